// hv_pdo.cu -- pseudo-differential operator probing (section 3.4, appendix A)
// and the low-rank-symbol PsiDO apply (section 3.3, eq. (lr-psido)):
//   H~ v = Re sum_k D_{a_k} F^-1 D_{b_k} F v
// with F the 2D DFT of the interior grid (cuFFT, complex-to-complex).
//
// Build: the probe v_p = sum_k exp(i x . xi_k) (r sample frequencies on a
// circle of radius rho0, snapped to DFT frequencies, +- pairs so v_p is
// real), one Hessian application, the DFT of H v_p, and per sample the
// spectrum inside a disc of radius rho0 sin(pi / r) around xi_k moved to the
// origin (demodulation) and transformed back: the symbol column a_k(x) =
// s(x, xi_k).  Weights b_k(xi) = (rho / rho_k) w_k(theta), w_k the
// trigonometric interpolation basis of the r nominal angles.
// The transposed apply B^T w = Re F^-1 sum_k conj(b_k) F (conj(a_k) w) and the
// square-root form of section 3.7 (columns sqrt(max(Re a_k, 0)), weights with
// radial order 1/2, approximation B B^T) live here too.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>

namespace hvk {

namespace {

__device__ __forceinline__ int signed_index(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// v_p(z, x) = sum_k cos(2 pi (iz_k z / nz + ix_k x / nx)) over the sample pairs,
// phases reduced exactly in integers (the probe is sum_k exp(i x . xi_k)).
__global__ void k_pdo_probe(float *v, LrGeo g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nz * g.nx) return;
    const int z = i / g.nx, x = i - z * g.nx;
    float s = 0.0f;
    for (int k = 0; k < g.r; ++k) {
        const long long pz = (((long long)g.iz[k] * z) % g.nz + g.nz) % g.nz;
        const long long px = (((long long)g.ix[k] * x) % g.nx + g.nx) % g.nx;
        const double ph = (double)pz / g.nz + (double)px / g.nx;   // in [0, 2)
        s += cospif((float)(2.0 * ph));
    }
    v[i] = s;
}

__global__ void k_real_to_complex(const float *__restrict__ v, float2 *__restrict__ c, size_t n, size_t n_pad)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) c[i] = make_float2(i < n ? v[i] : 0.0f, 0.0f);   // zero the unused vectors of a batch
}

// Y_k(i, j) = (U masked to the disc around xi_k)(i + iz_k, j + ix_k) / N: the
// separated, demodulated spectrum of column k (the window decision in FP64).
__global__ void k_pdo_separate(const float2 *__restrict__ U, float2 *__restrict__ Y, LrGeo g)
{
    const size_t N = (size_t)g.nz * g.nx;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)g.r * N) return;
    const int k = (int)(t / N);
    const int e = (int)(t - (size_t)k * N);
    const int i = e / g.nx, j = e - i * g.nx;
    const int si = ((i + g.iz[k]) % g.nz + g.nz) % g.nz, sj = ((j + g.ix[k]) % g.nx + g.nx) % g.nx;
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double fz = two_pi * ((double)signed_index(si, g.nz) / ((double)g.nz * g.h));
    const double fx = two_pi * ((double)signed_index(sj, g.nx) / ((double)g.nx * g.h));
    const double kz = two_pi * g.iz[k] / ((double)g.nz * g.h), kx = two_pi * g.ix[k] / ((double)g.nx * g.h);
    const bool in = hypot(fz - kz, fx - kx) < g.win;
    const float inv = 1.0f / (float)N;
    const float2 u = U[(size_t)si * g.nx + sj];
    Y[t] = in ? make_float2(u.x * inv, u.y * inv) : make_float2(0.0f, 0.0f);
}

// b_k(xi) = (rho / rho_k)^p (1/r) [1 + 2 sum_{m<r/2} cos(m (theta - theta_k)) + cos(r/2 (theta - theta_k))],
// p = 1 (the order of H_d) or 1/2 (its square root).
__global__ void k_pdo_weights(float2 *__restrict__ b, LrGeo g, bool half_order)
{
    const size_t N = (size_t)g.nz * g.nx;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)g.r * N) return;
    const int k = (int)(t / N);
    const int e = (int)(t - (size_t)k * N);
    const int i = e / g.nx, j = e - i * g.nx;
    const float two_pi = 6.283185307179586f, hf = (float)g.h;
    const float fz = two_pi * ((float)signed_index(i, g.nz) / ((float)g.nz * hf));
    const float fx = two_pi * ((float)signed_index(j, g.nx) / ((float)g.nx * hf));
    const float rho = hypotf(fz, fx);
    const float d = atan2f(fz, fx) - two_pi * k / g.r;
    float w = 1.0f;
    for (int m = 1; m < g.r / 2; ++m) w += 2.0f * cosf(m * d);
    w += cosf((g.r / 2) * d);
    const float radial = rho / g.rho[k];
    b[t] = make_float2((half_order ? sqrtf(radial) : radial) * (w / g.r), 0.0f);
}

// a <- (sqrt(max(Re a, 0)), 0): the symbol of the square root (section 3.7).
__global__ void k_sqrt_real(const float2 *in, float2 *out, size_t n)   // in == out allowed
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2(sqrtf(fmaxf(in[i].x, 0.0f)), 0.0f);
}

// The elementwise kernels of the apply index points by blockIdx.x (and the
// vector and term by blockIdx.y / blockIdx.z): no 64-bit division per element.

// Y[k][q] = b_k V_q / N for the r terms and the kb vectors of a batch (complex
// products); grid (points / 256, kb, r).
__global__ void k_lr_scale(const float2 *__restrict__ V, const float2 *__restrict__ b, float2 *__restrict__ Y, int r,
                           int kb, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int q = blockIdx.y, k = blockIdx.z;
    const size_t t = ((size_t)k * kb + q) * N + e;
    const float2 v = V[(size_t)q * N + e];
    const float2 w = b[(size_t)k * N + e];
    const float inv = 1.0f / (float)N;
    Y[t] = make_float2(fmaf(w.x, v.x, -w.y * v.y) * inv, fmaf(w.x, v.y, w.y * v.x) * inv);
}

// out_q = Re sum_k a_k y[k][q], summed in k order, for the nq valid vectors of a
// batch; grid (points / 256, nq).
__global__ void k_lr_combine(const float2 *__restrict__ A, const float2 *__restrict__ Y, float *__restrict__ out, int r,
                             int kb, int nq, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int q = blockIdx.y;
    const size_t t = (size_t)q * N + e;
    float s = 0.0f;
    for (int k = 0; k < r; ++k) {
        const float2 a = A[(size_t)k * N + e], y = Y[((size_t)k * kb + q) * N + e];
        s = fmaf(a.x, y.x, fmaf(-a.y, y.y, s));
    }
    out[t] = s;
}

// Transposed apply, first half: Y[k][q] = conj(a_k) w_q (complex times real);
// grid (points / 256, kb, r).
__global__ void k_lrT_premul(const float *__restrict__ w, const float2 *__restrict__ A, float2 *__restrict__ Y, int r,
                             int kb, int nq, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int q = blockIdx.y, k = blockIdx.z;
    const size_t t = ((size_t)k * kb + q) * N + e;
    const float x = q < nq ? w[(size_t)q * N + e] : 0.0f;
    const float2 a = A[(size_t)k * N + e];
    Y[t] = make_float2(a.x * x, -a.y * x);
}

// Transposed apply, second half: V_q = (1/N) sum_k conj(b_k) Y[k][q], in k
// order; grid (points / 256, kb).
__global__ void k_lrT_sum(const float2 *__restrict__ Y, const float2 *__restrict__ b, float2 *__restrict__ V, int r,
                          int kb, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int q = blockIdx.y;
    const size_t t = (size_t)q * N + e;
    float re = 0.0f, im = 0.0f;
    for (int k = 0; k < r; ++k) {
        const float2 w = b[(size_t)k * N + e], y = Y[((size_t)k * kb + q) * N + e];
        re = fmaf(w.x, y.x, fmaf(w.y, y.y, re));     // conj(w) y
        im = fmaf(w.x, y.y, fmaf(-w.y, y.x, im));
    }
    const float inv = 1.0f / (float)N;
    V[t] = make_float2(re * inv, im * inv);
}

__global__ void k_real_part(const float2 *__restrict__ V, float *__restrict__ out, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = V[i].x;
}

int check(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int cufft_check(cufftResult r, const char *what)
{
    if (r != CUFFT_SUCCESS) return hvi::fail(HV_ECUDA, "%s: cuFFT error %d", what, (int)r);
    return HV_OK;
}

}  // namespace

int lr_samples(int nz, int nx, double h, double rho0, int r, LrGeo &g)
{
    if (r < 2 || r % 2 || r > kLrMaxTerms) return hvi::fail(HV_EINVAL, "r = %d; need an even count in [2, %d]", r, kLrMaxTerms);
    if (!(rho0 > 0)) return hvi::fail(HV_EINVAL, "rho0 must be > 0");
    g.nz = nz;
    g.nx = nx;
    g.r = r;
    g.h = h;
    g.win = rho0 * std::sin(M_PI / r);
    if (rho0 + g.win >= M_PI / h)
        return hvi::fail(HV_EINVAL, "rho0 + window radius %g reaches the Nyquist frequency %g rad/m", rho0 + g.win, M_PI / h);
    const double dz = 2.0 * M_PI / (nz * h), dx = 2.0 * M_PI / (nx * h);
    for (int k = 0; k < r; ++k) {
        const double th = 2.0 * M_PI * k / r;
        g.iz[k] = (int)std::nearbyint(rho0 * std::sin(th) / dz);   // ties to even, as the oracle rounds
        g.ix[k] = (int)std::nearbyint(rho0 * std::cos(th) / dx);
        g.rho[k] = (float)std::hypot(g.iz[k] * dz, g.ix[k] * dx);
        if (g.iz[k] == 0 && g.ix[k] == 0) return hvi::fail(HV_EINVAL, "rho0 %g snaps to the zero frequency", rho0);
    }
    return HV_OK;
}

// Vectors per apply batch: up to 64, with the batch's r spectra within 256 MB
// (1 GB with the fused transforms, which need no library plan of r x kb
// transforms and its work area).
int lr_batch(const LrGeo &g, bool fused)
{
    const size_t per = (size_t)g.r * g.nz * g.nx * sizeof(float2);
    const size_t kb = per > 0 ? ((size_t)(fused ? 1024 : 256) << 20) / per : 1;
    return (int)std::max<size_t>(1, std::min<size_t>(64, kb));
}

int lr_create(LrSym &L, const LrGeo &g)
{
    L.g = g;
    L.mu = new std::mutex;
    L.fused = lr_fused_default() && lr_fused_supported(g.nz, g.nx);
    L.kb = lr_batch(g, L.fused);
    const size_t N = (size_t)g.nz * g.nx;
    const size_t nY = (size_t)g.r * std::max(L.kb, 1) * N;   // apply: r x kb spectra; build: r spectra
    cudaError_t e;
    if ((e = cudaMalloc(&L.a, (size_t)g.r * N * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&L.b, (size_t)g.r * N * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&L.Y, nY * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&L.V, (size_t)L.kb * N * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&L.T, (size_t)L.kb * N * sizeof(float))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "low-rank symbol buffers: %s", cudaGetErrorString(e));
    int n[2] = {g.nz, g.nx};
    HV_RT_INTERNAL(cufft_check(cufftPlan2d(&L.pf, g.nz, g.nx, CUFFT_C2C), "cufftPlan2d"));
    L.pf_ok = true;
    HV_RT_INTERNAL(cufft_check(cufftPlanMany(&L.pi, 2, n, nullptr, 1, (int)N, nullptr, 1, (int)N, CUFFT_C2C, g.r),
                               "cufftPlanMany"));
    L.pi_ok = true;
    HV_RT_INTERNAL(cufft_check(cufftPlanMany(&L.pfb, 2, n, nullptr, 1, (int)N, nullptr, 1, (int)N, CUFFT_C2C, L.kb),
                               "cufftPlanMany"));
    L.pfb_ok = true;
    if (L.fused) return lr_fused_init(L);
    HV_RT_INTERNAL(cufft_check(cufftPlanMany(&L.pib, 2, n, nullptr, 1, (int)N, nullptr, 1, (int)N, CUFFT_C2C,
                                             g.r * L.kb),
                               "cufftPlanMany"));
    L.pib_ok = true;
    return HV_OK;
}

void lr_destroy(LrSym &L)
{
    if (L.pf_ok) cufftDestroy(L.pf);
    if (L.pi_ok) cufftDestroy(L.pi);
    if (L.pfb_ok) cufftDestroy(L.pfb);
    if (L.pib_ok) cufftDestroy(L.pib);
    if (L.done) cudaEventDestroy(L.done);
    cudaFree(L.a);
    cudaFree(L.b);
    cudaFree(L.Y);
    cudaFree(L.V);
    cudaFree(L.T);
    cudaFree(L.tw);
    cudaFree(L.part);
    delete L.mu;
    L = LrSym{};
}

int launch_pdo_probe(const LrGeo &g, float *v, cudaStream_t st)
{
    k_pdo_probe<<<blocks_for((size_t)g.nz * g.nx, 256), 256, 0, st>>>(v, g);
    return check("k_pdo_probe");
}

// a_k from H v_p (real, [nz][nx]); uses L.V and L.Y as scratch.  Also fills b_k.
int pdo_columns(LrSym &L, const float *Hvp, cudaStream_t st)
{
    const LrGeo &g = L.g;
    const size_t N = (size_t)g.nz * g.nx;
    k_real_to_complex<<<blocks_for(N, 256), 256, 0, st>>>(Hvp, L.V, N, N);
    HV_RT_INTERNAL(check("k_real_to_complex"));
    std::lock_guard<std::mutex> lk(*L.mu);
    HV_RT_INTERNAL(cufft_check(cufftSetStream(L.pf, st), "cufftSetStream"));
    HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pf, (cufftComplex *)L.V, (cufftComplex *)L.V, CUFFT_FORWARD), "forward FFT"));
    k_pdo_separate<<<blocks_for((size_t)g.r * N, 256), 256, 0, st>>>(L.V, L.a, g);
    HV_RT_INTERNAL(check("k_pdo_separate"));
    HV_RT_INTERNAL(cufft_check(cufftSetStream(L.pi, st), "cufftSetStream"));
    HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pi, (cufftComplex *)L.a, (cufftComplex *)L.a, CUFFT_INVERSE), "inverse FFT"));
    k_pdo_weights<<<blocks_for((size_t)g.r * N, 256), 256, 0, st>>>(L.b, g, false);
    HV_RT_INTERNAL(check("k_pdo_weights"));
    cudaEventRecord(L.done, st);
    return HV_OK;
}

// One batch (nq <= kb vectors) of the forward apply B v = Re sum_k a_k F^-1 (b_k F v).
static int lr_batch_forward(LrSym &L, const float *v, int nq, float *out, cudaStream_t st)
{
    const LrGeo &g = L.g;
    const size_t N = (size_t)g.nz * g.nx;
    const int kb = L.kb;
    k_real_to_complex<<<blocks_for((size_t)kb * N, 256), 256, 0, st>>>(v, L.V, (size_t)nq * N, (size_t)kb * N);
    HV_RT_INTERNAL(check("k_real_to_complex"));
    HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pfb, (cufftComplex *)L.V, (cufftComplex *)L.V, CUFFT_FORWARD),
                               "forward FFT"));
    if (L.fused) return lr_fused_forward(L, L.V, nq, out, st);
    k_lr_scale<<<dim3(blocks_for(N, 256), kb, g.r), 256, 0, st>>>(L.V, L.b, L.Y, g.r, kb, N);
    HV_RT_INTERNAL(check("k_lr_scale"));
    HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pib, (cufftComplex *)L.Y, (cufftComplex *)L.Y, CUFFT_INVERSE),
                               "inverse FFT"));
    k_lr_combine<<<dim3(blocks_for(N, 256), nq), 256, 0, st>>>(L.a, L.Y, out, g.r, kb, nq, N);
    return check("k_lr_combine");
}

// One batch of the transposed apply B^T w = Re F^-1 sum_k conj(b_k) F (conj(a_k) w).
static int lr_batch_transpose(LrSym &L, const float *w, int nq, float *out, cudaStream_t st)
{
    const LrGeo &g = L.g;
    const size_t N = (size_t)g.nz * g.nx;
    const int kb = L.kb;
    if (L.fused) {
        HV_RT_INTERNAL(lr_fused_transpose(L, w, nq, L.V, st));
    } else {
        k_lrT_premul<<<dim3(blocks_for(N, 256), kb, g.r), 256, 0, st>>>(w, L.a, L.Y, g.r, kb, nq, N);
        HV_RT_INTERNAL(check("k_lrT_premul"));
        HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pib, (cufftComplex *)L.Y, (cufftComplex *)L.Y, CUFFT_FORWARD),
                                   "forward FFT"));
        k_lrT_sum<<<dim3(blocks_for(N, 256), kb), 256, 0, st>>>(L.Y, L.b, L.V, g.r, kb, N);
        HV_RT_INTERNAL(check("k_lrT_sum"));
    }
    HV_RT_INTERNAL(cufft_check(cufftExecC2C(L.pfb, (cufftComplex *)L.V, (cufftComplex *)L.V, CUFFT_INVERSE),
                               "inverse FFT"));
    k_real_part<<<blocks_for((size_t)nq * N, 256), 256, 0, st>>>(L.V, out, (size_t)nq * N);
    return check("k_real_part");
}

int lr_apply(LrSym &L, const float *v, int k, float *out, cudaStream_t st, int op)
{
    const LrGeo &g = L.g;
    const size_t N = (size_t)g.nz * g.nx;
    // The object's scratch is shared: applies from different streams run one after another.
    std::lock_guard<std::mutex> lk(*L.mu);
    cudaError_t e = cudaStreamWaitEvent(st, L.done, 0);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
    HV_RT_INTERNAL(cufft_check(cufftSetStream(L.pfb, st), "cufftSetStream"));
    if (L.pib_ok) HV_RT_INTERNAL(cufft_check(cufftSetStream(L.pib, st), "cufftSetStream"));
    const int kb = L.kb;
    for (int j0 = 0; j0 < k; j0 += kb) {            // batches of kb vectors (the last one zero-padded)
        const int nq = std::min(kb, k - j0);
        const float *vj = v + (size_t)j0 * N;
        float *oj = out + (size_t)j0 * N;
        if (op == kLrForward) {
            HV_RT_INTERNAL(lr_batch_forward(L, vj, nq, oj, st));
        } else if (op == kLrTranspose) {
            HV_RT_INTERNAL(lr_batch_transpose(L, vj, nq, oj, st));
        } else {                                     // B B^T
            HV_RT_INTERNAL(lr_batch_transpose(L, vj, nq, L.T, st));
            HV_RT_INTERNAL(lr_batch_forward(L, L.T, nq, oj, st));
        }
    }
    e = cudaEventRecord(L.done, st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    return HV_OK;
}

// The square-root PDO approximation (section 3.7) of the PDO approximation src.
int pdo_sqrt(const LrSym &src, LrSym &out, cudaStream_t st)
{
    HV_RT_INTERNAL(lr_create(out, src.g));
    out.spd = true;
    cudaError_t e = cudaStreamWaitEvent(st, src.done, 0);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
    const size_t n = (size_t)src.g.r * src.g.nz * src.g.nx;
    k_sqrt_real<<<blocks_for(n, 256), 256, 0, st>>>(src.a, out.a, n);
    HV_RT_INTERNAL(check("k_sqrt_real"));
    k_pdo_weights<<<blocks_for(n, 256), 256, 0, st>>>(out.b, out.g, true);
    HV_RT_INTERNAL(check("k_pdo_weights"));
    e = cudaEventRecord(out.done, st);
    if (e == cudaSuccess) e = cudaEventRecord(src.done, st);   // destroying src now waits for the copy
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    return HV_OK;
}

void launch_sqrt_real(const float2 *in, float2 *out, size_t n, cudaStream_t st)
{
    k_sqrt_real<<<blocks_for(n, 256), 256, 0, st>>>(in, out, n);
    count_launch();
}

}  // namespace hvk
