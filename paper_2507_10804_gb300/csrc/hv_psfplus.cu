// hv_psfplus.cu -- the PSF+ low-rank symbol (section 3.6).
//
//  1. Symbol rows from the PSFs (section 3.5): s(x_k, xi) = sum_d p_k(d) e^{i xi . d},
//     the conjugated DFT of each PSF placed at the origin of the grid (r rows).
//  2. The SVD of the rows through their Gram matrix G = S S^H = U Lambda U^H
//     (FP64; Hermitian Jacobi on the host): the
//     basis B = Sigma^-1 U^H S of the r' dominant directions (sigma_i >=
//     tol sigma_1, at most 32) and A0 = W U Sigma, W the PSF lattice weights.
//  3. The refinement against the PDO columns S~_c at the PDO samples I_c:
//     A = (S~_c B_c^H + alpha A0)(B_c B_c^H + alpha I)^-1,
//     alpha = ||B_c||_F^2 / ||B||_F^2 (= ||B_c||_F^2 / r', B has orthonormal rows).
// The result is applied by the low-rank-symbol engine (hv_pdo.cu) with a_i =
// A[:, i], b_i = B[i].  The square-root form (section 3.7) replaces the rows
// and the PDO columns by sqrt(max(Re s, 0)) before step 2; it is applied as
// B B^T.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace hvk {

namespace {

using cd = std::complex<double>;
constexpr int kMaxPsfPlusRows = 256;   // PSFs whose Gram matrix the host eigensolver takes

// E[k][(dz mod nz) * nx + (dx mod nx)] = p_k(dz, dx) (E zeroed before).
__global__ void k_embed_psfs(const float *__restrict__ psf, float2 *__restrict__ E, int r, int R, int nz, int nx)
{
    const int W = 2 * R + 1;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)r * W * W) return;
    const int k = (int)(i / ((size_t)W * W));
    const int rem = (int)(i - (size_t)k * W * W);
    const int dz = rem / W - R, dx = rem % W - R;
    const int z = ((dz % nz) + nz) % nz, x = ((dx % nx) + nx) % nx;
    E[(size_t)k * nz * nx + (size_t)z * nx + x] = make_float2(psf[i], 0.0f);
}

__global__ void k_conj(float2 *__restrict__ a, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i].y = -a[i].y;
}

// G[i][j] = sum_e S[i][e] conj(S[j][e]) in FP64; one CTA per (i, j), j >= i.
__global__ void k_gram(const float2 *__restrict__ S, double2 *__restrict__ G, int r, size_t N)
{
    const int i = blockIdx.x, j = blockIdx.y;
    if (j < i) return;
    const float2 *a = S + (size_t)i * N, *b = S + (size_t)j * N;
    double re = 0.0, im = 0.0;                       // FP64: the small eigenvalues decide the rank
    for (size_t e = threadIdx.x; e < N; e += blockDim.x) {
        const float2 x = a[e], y = b[e];
        re = fma((double)x.x, (double)y.x, fma((double)x.y, (double)y.y, re));    // x conj(y)
        im = fma((double)x.y, (double)y.x, fma(-(double)x.x, (double)y.y, im));
    }
    __shared__ double sre[256], sim[256];
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sre[threadIdx.x] += sre[threadIdx.x + h];
            sim[threadIdx.x] += sim[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        G[(size_t)i * r + j] = make_double2(sre[0], sim[0]);
        G[(size_t)j * r + i] = make_double2(sre[0], -sim[0]);
    }
}

// B[i][e] = (1 / sigma_i) sum_k conj(U[k][i]) S[k][e].
__global__ void k_basis(const float2 *__restrict__ S, const double2 *__restrict__ U, const double *__restrict__ sig,
                        float2 *__restrict__ B, int r, int rr, size_t N)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)rr * N) return;
    const int i = (int)(t / N);
    const size_t e = t - (size_t)i * N;
    double re = 0.0, im = 0.0;                       // FP64: U^H S cancels to sigma_i << |S|
    for (int k = 0; k < r; ++k) {
        const double2 u = U[(size_t)k * rr + i];
        const float2 s = S[(size_t)k * N + e];
        re = fma(u.x, (double)s.x, fma(u.y, (double)s.y, re));     // conj(u) s
        im = fma(u.x, (double)s.y, fma(-u.y, (double)s.x, im));
    }
    B[t] = make_float2((float)(re / sig[i]), (float)(im / sig[i]));
}

// Bilinear lattice weights along one axis, as the PSF apply computes them.
__device__ __forceinline__ void lattice_axis(int i, int c0, int S, int n, int &a0, int &a1, float &f)
{
    int q = i - c0;
    q = max(q, 0);
    q = min(q, (n - 1) * S);
    a0 = min(q / S, max(n - 2, 0));
    a1 = min(a0 + 1, n - 1);
    f = (float)(q - a0 * S) / (float)S;
}

// A0[i][x] = sigma_i sum_k w_k(x) U[k][i].
__global__ void k_a0(const double2 *__restrict__ U, const double *__restrict__ sig, float2 *__restrict__ A0, PsfGeo pg,
                     int rr)
{
    const size_t N = (size_t)pg.nz * pg.nx;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)rr * N) return;
    const int i = (int)(t / N);
    const int e = (int)(t - (size_t)i * N);
    const int iz = e / pg.nx, ix = e - iz * pg.nx;
    int a[2], b[2];
    float fz, fx;
    lattice_axis(iz, pg.cz0, pg.S, pg.na, a[0], a[1], fz);
    lattice_axis(ix, pg.cx0, pg.S, pg.nb, b[0], b[1], fx);
    const float wa[2] = {1.0f - fz, fz}, wb[2] = {1.0f - fx, fx};
    double re = 0.0, im = 0.0;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            const float w = wa[p] * wb[q];
            if (w == 0.0f) continue;
            const double2 u = U[(size_t)(a[p] * pg.nb + b[q]) * rr + i];
            re = fma((double)w, u.x, re);
            im = fma((double)w, u.y, im);
        }
    A0[t] = make_float2((float)(re * sig[i]), (float)(im * sig[i]));
}

// Bc[i][c] = B[i][I_c].
__global__ void k_gather_cols(const float2 *__restrict__ B, const int *__restrict__ Ic, float2 *__restrict__ Bc,
                              int rr, int rc, size_t N)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rr * rc) return;
    const int i = t / rc, c = t - i * rc;
    Bc[t] = B[(size_t)i * N + Ic[c]];
}

// A[j][x] = sum_i (sum_c S~_c(x) conj(Bc[i][c]) + alpha A0[i][x]) Minv[i][j].
__global__ void k_refine(const float2 *__restrict__ Sc, const float2 *__restrict__ Bc, const float2 *__restrict__ A0,
                         const float2 *__restrict__ Minv, float alpha, float2 *__restrict__ A, int rr, int rc, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    float2 y[32];
    for (int i = 0; i < rr; ++i) {
        float re = alpha * A0[(size_t)i * N + e].x, im = alpha * A0[(size_t)i * N + e].y;
        for (int c = 0; c < rc; ++c) {
            const float2 s = Sc[(size_t)c * N + e], b = Bc[i * rc + c];
            re = fmaf(s.x, b.x, fmaf(s.y, b.y, re));   // s conj(b)
            im = fmaf(s.y, b.x, fmaf(-s.x, b.y, im));
        }
        y[i] = make_float2(re, im);
    }
    for (int j = 0; j < rr; ++j) {
        float re = 0.0f, im = 0.0f;
        for (int i = 0; i < rr; ++i) {
            const float2 m = Minv[i * rr + j];
            re = fmaf(y[i].x, m.x, fmaf(-y[i].y, m.y, re));
            im = fmaf(y[i].x, m.y, fmaf(y[i].y, m.x, im));
        }
        A[(size_t)j * N + e] = make_float2(re, im);
    }
}

unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

// Device scratch freed on every exit path.
struct Scratch {
    std::vector<void *> p;
    template <class T>
    int get(T **out, size_t bytes)
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(out), bytes);
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "PSF+ scratch: %s", cudaGetErrorString(e));
        p.push_back(*out);
        return HV_OK;
    }
    ~Scratch()
    {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

int build_psfplus(const PsfGeo &pg, const float *psf, const LrSym &pdo, double tol, bool spd, LrSym &out,
                  cudaStream_t st)
{
    const int r = pg.na * pg.nb, nz = pg.nz, nx = pg.nx, W = 2 * pg.R + 1, rc = pdo.g.r;
    const size_t N = (size_t)nz * nx;
    if (r > kMaxPsfPlusRows) return hvi::fail(HV_EINVAL, "PSF+ takes at most %d PSFs (%d given)", kMaxPsfPlusRows, r);
    if (W > nz || W > nx) return hvi::fail(HV_EINVAL, "PSF window %d wider than the %d x %d grid", W, nz, nx);
    if (!(tol > 0 && tol < 1)) return hvi::fail(HV_EINVAL, "rank tolerance %g; need 0 < tol < 1", tol);
    cudaError_t e = cudaStreamWaitEvent(st, pdo.done, 0);   // the PDO columns may come from another stream
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
    Scratch sc;
    float2 *S = nullptr;
    double2 *G = nullptr;
    HV_RT_INTERNAL(sc.get(&S, (size_t)r * N * sizeof(float2)));
    HV_RT_INTERNAL(sc.get(&G, (size_t)r * r * sizeof(double2)));
    // 1. rows
    e = cudaMemsetAsync(S, 0, (size_t)r * N * sizeof(float2), st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    k_embed_psfs<<<nblk((size_t)r * W * W, 256), 256, 0, st>>>(psf, S, r, pg.R, nz, nx);
    HV_RT_INTERNAL(launched("k_embed_psfs"));
    cufftHandle plan;
    int n[2] = {nz, nx};
    if (cufftPlanMany(&plan, 2, n, nullptr, 1, (int)N, nullptr, 1, (int)N, CUFFT_C2C, r) != CUFFT_SUCCESS)
        return hvi::fail(HV_ECUDA, "cufftPlanMany failed");
    cufftResult fr = cufftSetStream(plan, st);
    if (fr == CUFFT_SUCCESS) fr = cufftExecC2C(plan, (cufftComplex *)S, (cufftComplex *)S, CUFFT_FORWARD);
    cufftDestroy(plan);
    if (fr != CUFFT_SUCCESS) return hvi::fail(HV_ECUDA, "PSF row transforms: cuFFT error %d", (int)fr);
    k_conj<<<nblk((size_t)r * N, 256), 256, 0, st>>>(S, (size_t)r * N);
    HV_RT_INTERNAL(launched("k_conj"));
    const float2 *cols = pdo.a;
    if (spd) {   // section 3.7: rows and columns of the square root, sqrt(max(Re s, 0))
        float2 *sc_cols = nullptr;
        HV_RT_INTERNAL(sc.get(&sc_cols, (size_t)rc * N * sizeof(float2)));
        launch_sqrt_real(S, S, (size_t)r * N, st);
        launch_sqrt_real(pdo.a, sc_cols, (size_t)rc * N, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "k_sqrt_real: %s", cudaGetErrorString(e));
        cols = sc_cols;
    }
    // 2. Gram matrix, eigen-decomposition on the host, basis and A0
    k_gram<<<dim3(r, r), 256, 0, st>>>(S, G, r, N);
    HV_RT_INTERNAL(launched("k_gram"));
    std::vector<double2> Gh((size_t)r * r);
    e = cudaMemcpyAsync(Gh.data(), G, Gh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "PSF+ Gram matrix: %s", cudaGetErrorString(e));
    std::vector<cd> Gc((size_t)r * r), V;
    for (size_t i = 0; i < Gc.size(); ++i) Gc[i] = cd(Gh[i].x, Gh[i].y);
    std::vector<double> lam;
    HV_RT_INTERNAL(hvi::hermitian_eig(r, Gc, lam, V));
    const double s1 = std::sqrt(std::max(lam[0], 0.0));
    if (!(s1 > 0)) return hvi::fail(HV_EINVAL, "PSF+: the PSFs are all zero");
    int rr = 0;
    while (rr < r && rr < kLrMaxTerms && std::sqrt(std::max(lam[rr], 0.0)) >= tol * s1) ++rr;
    std::vector<double2> Uh((size_t)r * rr);
    std::vector<double> sig(rr);
    for (int i = 0; i < rr; ++i) sig[i] = std::sqrt(lam[i]);
    for (int k = 0; k < r; ++k)
        for (int i = 0; i < rr; ++i) Uh[(size_t)k * rr + i] = make_double2(V[(size_t)k * r + i].real(),
                                                                          V[(size_t)k * r + i].imag());
    double2 *Ud = nullptr;
    float2 *A0 = nullptr, *Bc = nullptr, *Minvd = nullptr;
    double *sigd = nullptr;
    int *Icd = nullptr;
    HV_RT_INTERNAL(sc.get(&Ud, Uh.size() * sizeof(double2)));
    HV_RT_INTERNAL(sc.get(&sigd, rr * sizeof(double)));
    HV_RT_INTERNAL(sc.get(&A0, (size_t)rr * N * sizeof(float2)));
    HV_RT_INTERNAL(sc.get(&Bc, (size_t)rr * rc * sizeof(float2)));
    HV_RT_INTERNAL(sc.get(&Minvd, (size_t)rr * rr * sizeof(float2)));
    HV_RT_INTERNAL(sc.get(&Icd, rc * sizeof(int)));
    std::vector<int> Ic(rc);
    for (int c = 0; c < rc; ++c) Ic[c] = ((pdo.g.iz[c] % nz + nz) % nz) * nx + ((pdo.g.ix[c] % nx + nx) % nx);
    if ((e = cudaMemcpyAsync(Ud, Uh.data(), Uh.size() * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sigd, sig.data(), rr * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(Icd, Ic.data(), rc * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "PSF+ uploads: %s", cudaGetErrorString(e));
    LrGeo g;
    g.nz = nz;
    g.nx = nx;
    g.r = rr;
    g.h = pdo.g.h;
    HV_RT_INTERNAL(lr_create(out, g));
    out.spd = spd;
    k_basis<<<nblk((size_t)rr * N, 256), 256, 0, st>>>(S, Ud, sigd, out.b, r, rr, N);
    HV_RT_INTERNAL(launched("k_basis"));
    k_a0<<<nblk((size_t)rr * N, 256), 256, 0, st>>>(Ud, sigd, A0, pg, rr);
    HV_RT_INTERNAL(launched("k_a0"));
    // 3. refinement against the PDO columns
    k_gather_cols<<<nblk((size_t)rr * rc, 128), 128, 0, st>>>(out.b, Icd, Bc, rr, rc, N);
    HV_RT_INTERNAL(launched("k_gather_cols"));
    std::vector<float2> Bch((size_t)rr * rc);
    e = cudaMemcpyAsync(Bch.data(), Bc, Bch.size() * sizeof(float2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "PSF+ columns of the basis: %s", cudaGetErrorString(e));
    double bc2 = 0.0;
    for (const float2 &b : Bch) bc2 += (double)b.x * b.x + (double)b.y * b.y;
    const double alpha = bc2 / rr;
    std::vector<cd> M((size_t)rr * rr), Minv;
    for (int i = 0; i < rr; ++i)
        for (int j = 0; j < rr; ++j) {
            cd s = (i == j) ? cd(alpha, 0.0) : cd(0.0, 0.0);
            for (int c = 0; c < rc; ++c)
                s += cd(Bch[(size_t)i * rc + c].x, Bch[(size_t)i * rc + c].y) *
                     std::conj(cd(Bch[(size_t)j * rc + c].x, Bch[(size_t)j * rc + c].y));
            M[(size_t)i * rr + j] = s;
        }
    HV_RT_INTERNAL(hvi::small_inverse(rr, M, Minv));
    std::vector<float2> Mh((size_t)rr * rr);
    for (size_t i = 0; i < Mh.size(); ++i) Mh[i] = make_float2((float)Minv[i].real(), (float)Minv[i].imag());
    e = cudaMemcpyAsync(Minvd, Mh.data(), Mh.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "PSF+ upload: %s", cudaGetErrorString(e));
    k_refine<<<nblk(N, 128), 128, 0, st>>>(cols, Bc, A0, Minvd, (float)alpha, out.a, rr, rc, N);
    HV_RT_INTERNAL(launched("k_refine"));
    e = cudaStreamSynchronize(st);   // the scratch is freed on return
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "PSF+ build: %s", cudaGetErrorString(e));
    cudaEventRecord(out.done, st);
    return HV_OK;
}

}  // namespace hvk
