// hv_lrfft.cu -- the library's own 2D DFTs for the low-rank-symbol applies of
// sections 3.3-3.7,
//   B v    = Re sum_k a_k F^-1 (b_k F v)                  (eq. (lr-psido))
//   B^T w  = Re F^-1 sum_k conj(b_k) F (conj(a_k) w),
// with the symbol products fused into the transforms.  The r-term spectra
// exist only once, between the column pass and the row pass of each 2D
// transform (written once, read once), instead of being written by a product
// kernel, read and written twice by a library 2D transform and read again by a
// combining kernel.
//
// Each 1D DFT of length L = R1 R2 (a power of two, 16..512) is the four-step
// factorisation: with n = n1 + R1 n2 and k = k2 + R2 k1,
//   X[k2 + R2 k1] = sum_n1 W_R1^(n1 k1) W_L^(n1 k2) sum_n2 x[n1 + R1 n2] W_R2^(n2 k2),
// W_M = exp(-2 pi i / M) (forward; conjugated for the inverse).  Thread n1 of a
// sequence holds x[n1 + R1 n2] in registers and does the length-R2 DFT there
// (radix 2), multiplies by W_L^(n1 k2) and passes the values through shared
// memory to thread k2, which does the length-R1 DFT.  A CTA works on S
// sequences at once: S rows (a row's elements contiguous), or S adjacent
// columns with the column index fastest across threads, so that every global
// access is a run of consecutive elements.  The twiddles are tables computed
// in FP64 on the host and rounded once.  The transforms are unnormalised, as
// the library's FFT convention; the 1/N of the applies is applied where the
// cuFFT path applies it.
#include "hv_internal.h"

#include <cmath>
#include <mutex>
#include <vector>

namespace hvk {

namespace {

__constant__ float2 c_w32[32];   // exp(-2 pi i j / 32)

template <int R>
__host__ __device__ constexpr int bitrev(int i)
{
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// b = w v for the twiddle w = exp(-+2 pi i m / 32) of a radix-2 butterfly; m is
// a constant once the loops are unrolled, so the multiplications by 1, -+i and
// the odd multiples of pi / 4 reduce to sign changes, swaps and one scale.
template <bool INV>
__device__ __forceinline__ float2 twiddle32(int m, float2 x)
{
    constexpr float c = 0.70710678118654752f;   // 1 / sqrt(2)
    if (m == 0) return x;
    if (m == 8) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    if (m == 4) return INV ? make_float2(c * (x.x - x.y), c * (x.x + x.y)) : make_float2(c * (x.x + x.y), c * (x.y - x.x));
    if (m == 12)
        return INV ? make_float2(-c * (x.x + x.y), c * (x.x - x.y)) : make_float2(c * (x.y - x.x), -c * (x.x + x.y));
    float2 w = c_w32[m];
    if (INV) w.y = -w.y;
    return cmul(w, x);
}

// In-register DFT of length R (2..32): radix-2 decimation in time after a
// bit-reversal permutation; INV conjugates the twiddles.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R])
{
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = bitrev<R>(i);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int half = 1; half < R; half <<= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * half) {
#pragma unroll
            for (int p = 0; p < half; ++p) {
                // exp(-2 pi i p / (2 half)) v = W_32^(p 16 / half) v
                const float2 a = v[g + p], b = twiddle32<INV>(p * (16 / half), v[g + p + half]);
                v[g + p] = make_float2(a.x + b.x, a.y + b.y);
                v[g + p + half] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
}

template <int R1, int R2>
struct Split {
    static constexpr int TP = R1 > R2 ? R1 : R2;   // threads per sequence (length R1 R2)
};

// Step 1 of a sequence held by thread n1 (< R1): v[n2] = x[n1 + R1 n2] on entry;
// returns the twiddled length-R2 DFTs for thread k2 to pick up.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void step1(float2 (&v)[R2], int n1, const float2 *__restrict__ tw)
{
    dft_reg<R2, INV>(v);
#pragma unroll
    for (int k2 = 1; k2 < R2; ++k2) {
        float2 w = __ldg(tw + n1 * k2);
        if (INV) w.y = -w.y;
        v[k2] = cmul(v[k2], w);
    }
}

// ---- forward apply: columns.  T_k[q] = column DFT^-1 of (b_k V_q / N) for the
// terms of this CTA's chunk; grid (nx / S, nq, term chunks); thread = t S + s.
template <int R1, int R2, int S>
__global__ void __launch_bounds__(S *Split<R1, R2>::TP, R1 <= 16 ? 2 : 1) k_lrf_cols(const float2 *__restrict__ V,
                                                                   const float2 *__restrict__ B,
                                                                   const float2 *__restrict__ tw, float2 *__restrict__ T,
                                                                   int r, int kb, int nx, int kchunk)
{
    constexpr int L = R1 * R2;
    __shared__ float2 sY[R1][R2][S];
    const int s = threadIdx.x % S, t = threadIdx.x / S;
    const int c = blockIdx.x * S + s, q = blockIdx.y;
    const size_t N = (size_t)L * nx;
    const float inv = 1.0f / (float)N;
    // element n2 of this thread's part of the column: offset e0 + n2 * es (N < 2^31)
    const int e0 = t * nx + c, es = R1 * nx;
    const float2 *Vq = V + (size_t)q * N;   // read again for every term (from L1): registers are scarce
    const int k0 = blockIdx.z * kchunk, k1 = min(r, k0 + kchunk);
    for (int k = k0; k < k1; ++k) {
        if (t < R1) {
            const float2 *bk = B + (size_t)k * N;
            float2 v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) {   // b_k V / N, as the cuFFT path scales
                const int e = e0 + n2 * es;
                const float2 w = bk[e], x = __ldg(Vq + e);
                v[n2] = make_float2(fmaf(w.x, x.x, -w.y * x.y) * inv, fmaf(w.x, x.y, w.y * x.x) * inv);
            }
            step1<R1, R2, true>(v, t, tw);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) sY[t][k2][s] = v[k2];
        }
        __syncthreads();
        if (t < R2) {
            float2 u[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) u[n1] = sY[n1][t][s];
            dft_reg<R1, true>(u);
            float2 *Tk = T + ((size_t)k * kb + q) * N + (t * nx + c);
#pragma unroll
            for (int j = 0; j < R1; ++j) Tk[j * (R2 * nx)] = u[j];
        }
        __syncthreads();
    }
}

// ---- forward apply: rows.  out_q = Re sum_k a_k (row DFT^-1 of T_k[q]), summed
// in k order over the terms of this CTA's chunk; grid (nz / S, nq, term
// chunks); thread = s TP + t.  With one chunk the sum goes to out[q], else to
// part[chunk][q] for k_sum_real.
template <int R1, int R2, int S>
__global__ void __launch_bounds__(S *Split<R1, R2>::TP) k_lrf_rows(const float2 *__restrict__ T,
                                                                   const float2 *__restrict__ A,
                                                                   const float2 *__restrict__ tw, float *__restrict__ out,
                                                                   float *__restrict__ part, int r, int kb, int nz,
                                                                   int kchunk)
{
    constexpr int L = R1 * R2, TP = Split<R1, R2>::TP;
    __shared__ float2 sY[S][R1][R2 + 1];
    const int s = threadIdx.x / TP, t = threadIdx.x % TP;
    const int z = blockIdx.x * S + s, q = blockIdx.y;
    const size_t N = (size_t)nz * L, row = (size_t)z * L;
    float acc[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) acc[j] = 0.0f;
    const int k0 = blockIdx.z * kchunk, k1 = min(r, k0 + kchunk);
    for (int k = k0; k < k1; ++k) {
        if (t < R1) {
            const float2 *Tk = T + ((size_t)k * kb + q) * N + row;
            float2 v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) v[n2] = Tk[t + R1 * n2];
            step1<R1, R2, true>(v, t, tw);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) sY[s][t][k2] = v[k2];
        }
        __syncthreads();
        if (t < R2) {
            float2 u[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) u[n1] = sY[s][n1][t];
            dft_reg<R1, true>(u);
            const float2 *ak = A + (size_t)k * N + row;
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const float2 a = ak[t + R2 * j];
                acc[j] = fmaf(a.x, u[j].x, fmaf(-a.y, u[j].y, acc[j]));
            }
        }
        __syncthreads();
    }
    float *dst = gridDim.z == 1 ? out + (size_t)q * N : part + ((size_t)blockIdx.z * gridDim.y + q) * N;
    if (t < R2)
#pragma unroll
        for (int j = 0; j < R1; ++j) dst[row + t + R2 * j] = acc[j];
}

// ---- transposed apply: rows.  T_k[q] = row DFT of conj(a_k) w_q for the terms
// of this CTA's chunk; grid (nz / S, nq, term chunks); thread = s TP + t.
template <int R1, int R2, int S>
__global__ void __launch_bounds__(S *Split<R1, R2>::TP) k_lrt_rows(const float *__restrict__ Wv,
                                                                   const float2 *__restrict__ A,
                                                                   const float2 *__restrict__ tw, float2 *__restrict__ T,
                                                                   int r, int kb, int nz, int kchunk)
{
    constexpr int L = R1 * R2, TP = Split<R1, R2>::TP;
    __shared__ float2 sY[S][R1][R2 + 1];
    const int s = threadIdx.x / TP, t = threadIdx.x % TP;
    const int z = blockIdx.x * S + s, q = blockIdx.y;
    const size_t N = (size_t)nz * L, row = (size_t)z * L;
    float win[R2];
    if (t < R1)
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) win[n2] = Wv[(size_t)q * N + row + t + R1 * n2];
    const int k0 = blockIdx.z * kchunk, k1 = min(r, k0 + kchunk);
    for (int k = k0; k < k1; ++k) {
        if (t < R1) {
            const float2 *ak = A + (size_t)k * N + row;
            float2 v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) {   // conj(a_k) w
                const float2 a = ak[t + R1 * n2];
                v[n2] = make_float2(a.x * win[n2], -a.y * win[n2]);
            }
            step1<R1, R2, false>(v, t, tw);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) sY[s][t][k2] = v[k2];
        }
        __syncthreads();
        if (t < R2) {
            float2 u[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) u[n1] = sY[s][n1][t];
            dft_reg<R1, false>(u);
            float2 *Tk = T + ((size_t)k * kb + q) * N + row;
#pragma unroll
            for (int j = 0; j < R1; ++j) Tk[t + R2 * j] = u[j];
        }
        __syncthreads();
    }
}

// ---- transposed apply: columns.  V_q = (1/N) sum_k conj(b_k) (column DFT of
// T_k[q]), summed in k order over the terms of this CTA's chunk; grid (nx / S,
// nq, term chunks); thread = t S + s.  With one chunk the scaled sum goes to
// V[q], else the unscaled one to part[chunk][q] for k_sum_cplx.
template <int R1, int R2, int S>
__global__ void __launch_bounds__(S *Split<R1, R2>::TP, R1 <= 16 ? 2 : 1) k_lrt_cols(const float2 *__restrict__ T,
                                                                   const float2 *__restrict__ B,
                                                                   const float2 *__restrict__ tw, float2 *__restrict__ V,
                                                                   float2 *__restrict__ part, int r, int kb, int nx,
                                                                   int kchunk)
{
    constexpr int L = R1 * R2;
    __shared__ float2 sY[R1][R2][S];
    const int s = threadIdx.x % S, t = threadIdx.x / S;
    const int c = blockIdx.x * S + s, q = blockIdx.y;
    const size_t N = (size_t)L * nx;
    float re[R1], im[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) re[j] = im[j] = 0.0f;
    const int k0 = blockIdx.z * kchunk, k1 = min(r, k0 + kchunk);
    for (int k = k0; k < k1; ++k) {
        if (t < R1) {
            const float2 *Tk = T + ((size_t)k * kb + q) * N + (t * nx + c);
            float2 v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) v[n2] = Tk[n2 * (R1 * nx)];
            step1<R1, R2, false>(v, t, tw);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) sY[t][k2][s] = v[k2];
        }
        __syncthreads();
        if (t < R2) {
            float2 u[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) u[n1] = sY[n1][t][s];
            dft_reg<R1, false>(u);
            const float2 *bk = B + (size_t)k * N + (t * nx + c);
#pragma unroll
            for (int j = 0; j < R1; ++j) {   // conj(b_k) y, as the cuFFT path sums
                const float2 w = bk[j * (R2 * nx)];
                re[j] = fmaf(w.x, u[j].x, fmaf(w.y, u[j].y, re[j]));
                im[j] = fmaf(w.x, u[j].y, fmaf(-w.y, u[j].x, im[j]));
            }
        }
        __syncthreads();
    }
    const bool one = gridDim.z == 1;
    const float inv = one ? 1.0f / (float)N : 1.0f;
    float2 *dst = one ? V + (size_t)q * N : part + ((size_t)blockIdx.z * gridDim.y + q) * N;
    if (t < R2)
#pragma unroll
        for (int j = 0; j < R1; ++j) dst[(t * nx + c) + j * (R2 * nx)] = make_float2(re[j] * inv, im[j] * inv);
}

// out[q][e] = sum_c part[c][q][e] in chunk order; grid (N / 256, nq).
__global__ void k_sum_real(const float *__restrict__ part, float *__restrict__ out, int nc, int nq, int N)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (e >= N) return;
    float s = 0.0f;
    for (int c = 0; c < nc; ++c) s += part[((size_t)c * nq + q) * N + e];
    out[(size_t)q * N + e] = s;
}

// V[q][e] = (1/N) sum_c part[c][q][e] in chunk order; grid (N / 256, nq).
__global__ void k_sum_cplx(const float2 *__restrict__ part, float2 *__restrict__ V, int nc, int nq, int N)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (e >= N) return;
    float re = 0.0f, im = 0.0f;
    for (int c = 0; c < nc; ++c) {
        const float2 v = part[((size_t)c * nq + q) * N + e];
        re += v.x;
        im += v.y;
    }
    const float inv = 1.0f / (float)N;
    V[(size_t)q * N + e] = make_float2(re * inv, im * inv);
}

// Runs f(Split<R1, R2>{}, S-tag) for a supported length, else returns HV_ENOTSUP.
template <int V_>
struct Int {
    static constexpr int value = V_;
};
template <class F>
int with_split(int L, F &&f)
{
    switch (L) {
    case 16: return f(Int<4>{}, Int<4>{}, Int<16>{});
    case 32: return f(Int<8>{}, Int<4>{}, Int<16>{});
    case 64: return f(Int<8>{}, Int<8>{}, Int<16>{});
    case 128: return f(Int<16>{}, Int<8>{}, Int<16>{});
    case 256: return f(Int<16>{}, Int<16>{}, Int<16>{});
    case 512: return f(Int<32>{}, Int<16>{}, Int<8>{});
    default: return HV_ENOTSUP;
    }
}

bool supported(int L) { return L >= 16 && L <= 512 && (L & (L - 1)) == 0; }

int launched(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

constexpr int kTermChunk = 4;   // terms per CTA in the passes that write T
constexpr int kSumChunk = 8;    // terms per CTA in the passes that sum over the terms

std::mutex g_mu;
bool g_fused_default = true;

}  // namespace

bool lr_fused_default()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_fused_default;
}

bool lr_fused_supported(int nz, int nx) { return supported(nz) && supported(nx); }

int lr_fused_init(LrSym &L)
{
    const int nz = L.g.nz, nx = L.g.nx;
    std::vector<float2> h(32 + nz + nx);
    auto fill = [](float2 *p, int n) {
        for (int m = 0; m < n; ++m) {
            const double a = -2.0 * M_PI * (double)m / (double)n;
            p[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    };
    fill(h.data(), 32);
    fill(h.data() + 32, nz);
    fill(h.data() + 32 + nz, nx);
    const int nc = (L.g.r + kSumChunk - 1) / kSumChunk;   // partial sums of the term chunks
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_w32, h.data(), 32 * sizeof(float2))) != cudaSuccess ||
        (nc > 1 && (e = cudaMalloc(&L.part, (size_t)nc * L.kb * nz * nx * sizeof(float2))) != cudaSuccess) ||
        (e = cudaMalloc(&L.tw, (size_t)(nz + nx) * sizeof(float2))) != cudaSuccess ||
        (e = cudaMemcpy(L.tw, h.data() + 32, (size_t)(nz + nx) * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "fused transform tables: %s", cudaGetErrorString(e));
    return HV_OK;
}

int lr_fused_forward(const LrSym &L, const float2 *V, int nq, float *out, cudaStream_t st)
{
    const LrGeo &g = L.g;
    const float2 *twz = L.tw, *twx = L.tw + g.nz;
    int rc = with_split(g.nz, [&](auto r1, auto r2, auto sz) -> int {
        constexpr int R1 = decltype(r1)::value, R2 = decltype(r2)::value, S = decltype(sz)::value;
        const dim3 grid(g.nx / S, nq, (g.r + kTermChunk - 1) / kTermChunk);
        k_lrf_cols<R1, R2, S><<<grid, S * Split<R1, R2>::TP, 0, st>>>(V, L.b, twz, L.Y, g.r, L.kb, g.nx, kTermChunk);
        return launched("k_lrf_cols");
    });
    if (rc != HV_OK) return rc;
    const int nc = (g.r + kSumChunk - 1) / kSumChunk, N = g.nz * g.nx;
    float *part = reinterpret_cast<float *>(L.part);
    rc = with_split(g.nx, [&](auto r1, auto r2, auto sz) -> int {
        constexpr int R1 = decltype(r1)::value, R2 = decltype(r2)::value, S = decltype(sz)::value;
        k_lrf_rows<R1, R2, S><<<dim3(g.nz / S, nq, nc), S * Split<R1, R2>::TP, 0, st>>>(L.Y, L.a, twx, out, part,
                                                                                       g.r, L.kb, g.nz, kSumChunk);
        return launched("k_lrf_rows");
    });
    if (rc != HV_OK || nc == 1) return rc;
    k_sum_real<<<dim3((N + 255) / 256, nq), 256, 0, st>>>(part, out, nc, nq, N);
    return launched("k_sum_real");
}

int lr_fused_transpose(const LrSym &L, const float *w, int nq, float2 *V, cudaStream_t st)
{
    const LrGeo &g = L.g;
    const float2 *twz = L.tw, *twx = L.tw + g.nz;
    int rc = with_split(g.nx, [&](auto r1, auto r2, auto sz) -> int {
        constexpr int R1 = decltype(r1)::value, R2 = decltype(r2)::value, S = decltype(sz)::value;
        const dim3 grid(g.nz / S, nq, (g.r + kTermChunk - 1) / kTermChunk);
        k_lrt_rows<R1, R2, S><<<grid, S * Split<R1, R2>::TP, 0, st>>>(w, L.a, twx, L.Y, g.r, L.kb, g.nz, kTermChunk);
        return launched("k_lrt_rows");
    });
    if (rc != HV_OK) return rc;
    const int nc = (g.r + kSumChunk - 1) / kSumChunk, N = g.nz * g.nx;
    float2 *part = reinterpret_cast<float2 *>(L.part);
    rc = with_split(g.nz, [&](auto r1, auto r2, auto sz) -> int {
        constexpr int R1 = decltype(r1)::value, R2 = decltype(r2)::value, S = decltype(sz)::value;
        k_lrt_cols<R1, R2, S><<<dim3(g.nx / S, nq, nc), S * Split<R1, R2>::TP, 0, st>>>(L.Y, L.b, twz, V, part,
                                                                                       g.r, L.kb, g.nx, kSumChunk);
        return launched("k_lrt_cols");
    });
    if (rc != HV_OK || nc == 1) return rc;
    k_sum_cplx<<<dim3((N + 255) / 256, nq), 256, 0, st>>>(part, V, nc, nq, N);
    return launched("k_sum_cplx");
}

}  // namespace hvk

extern "C" int hv_set_fused_transforms(int enable)
{
    std::lock_guard<std::mutex> lk(hvk::g_mu);
    hvk::g_fused_default = enable != 0;
    return HV_OK;
}
