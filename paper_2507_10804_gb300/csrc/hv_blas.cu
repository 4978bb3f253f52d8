// hv_blas.cu -- skinny dense products over grid fields, shared by the
// low-rank, posterior and quadratic-model code:
//   rows_dot:  s[q]    = sum_e A[q][e] B[q][e]                 (k dot products)
//   coef:      C[q][j] = w[j] sum_e M[j][e] X[q][e]            (r x k dot products)
//   combine:   out[q][e] = base[q][e] + sign sum_j C[q][j] M[j][e]
// Reductions over the field run in chunks of kChunk points, one CTA per chunk
// and row, the chunks summed in a fixed order by a second kernel --
// deterministic, with the whole device busy even for a few long rows (one CTA
// per row left most SMs idle).  rows_dot keeps FP64 accuracy (it decides CG
// step lengths and gpCN acceptances) with double-float arithmetic on the FP32
// pipe inside a thread and FP64 above; coef sums in FP32 inside a chunk and
// FP64 across chunks (r x k dots: FP64 throughout would run at the FP64 rate).
// The sums over j in combine (at most 256 terms) run in FP32 with the
// coefficients rounded to FP32.
#include "hv_internal.h"

#include <algorithm>

namespace hvk {

namespace {

constexpr int kChunk = 2048;     // field points per CTA in the reductions
constexpr int kTile = 16;        // rows of M and of X per CTA in coef

unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    const double s = sh[0];
    __syncthreads();
    return s;
}

// part[q][c] = sum over chunk c of A[q][e] B[q][e]; grid (chunks, k), 256 threads.
__global__ void k_rows_dot_part(const float *__restrict__ A, const float *__restrict__ B, double *__restrict__ part,
                                size_t N, int nch)
{
    __shared__ double sh[256];
    const int c = blockIdx.x, q = blockIdx.y;
    const size_t o = (size_t)q * N, e0 = (size_t)c * kChunk, e1 = min(N, e0 + kChunk);
    // Double-float accumulation on the FP32 pipe (the FP64 pipe and its conversions are
    // slow on this part): each product is split exactly into p + pe (fmaf), the running
    // sum hi is kept with TwoSum, the rounding errors collect in lo; the thread's
    // partial hi + lo is then exact to about 2^-44 of the sum of |products|.
    float hi = 0.0f, lo = 0.0f;
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const float a = A[o + e], b = B[o + e];
        // explicit round-to-nearest intrinsics: no contraction may merge these steps
        const float p = __fmul_rn(a, b), pe = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p), bv = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv)), pe));
        hi = s;
    }
    const double t = block_sum((double)hi + (double)lo, sh);
    if (threadIdx.x == 0) part[(size_t)q * nch + c] = t;
}

// out[i] = scale * sum_c part[i][c] in chunk order (one thread per output).
__global__ void k_sum_parts(const double *__restrict__ part, double *__restrict__ out, int n, int nch, double scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(size_t)i * nch + c];
    out[i] = scale * s;
}

// part[(q * r + j) * nch + c] = sum over chunk c of M[j][e] X[q][e] for a
// kTile x kTile block of (j, q); grid (chunks, ceil(r / kTile), ceil(k / kTile)).
__global__ void k_coef_part(const float *__restrict__ M, const float *__restrict__ X, double *__restrict__ part, int r,
                            int k, size_t N, int nch)
{
    constexpr int kSub = 128;   // points staged per round
    __shared__ float sm[kTile][kSub + 1], sx[kTile][kSub + 1];
    const int c = blockIdx.x, j0 = blockIdx.y * kTile, q0 = blockIdx.z * kTile;
    const size_t e0 = (size_t)c * kChunk, e1 = min(N, e0 + kChunk);
    // thread t accumulates the pair (j0 + t / kTile, q0 + t % kTile); 256 threads = kTile^2 pairs
    const int tj = threadIdx.x / kTile, tq = threadIdx.x % kTile;
    float acc = 0.0f;
    for (size_t b = e0; b < e1; b += kSub) {
        const int n = (int)min((size_t)kSub, e1 - b);
        for (int i = threadIdx.x; i < kTile * kSub; i += blockDim.x) {
            const int row = i / kSub, col = i % kSub;
            const bool in = col < n;
            sm[row][col] = (in && j0 + row < r) ? M[(size_t)(j0 + row) * N + b + col] : 0.0f;
            sx[row][col] = (in && q0 + row < k) ? X[(size_t)(q0 + row) * N + b + col] : 0.0f;
        }
        __syncthreads();
        for (int col = 0; col < n; ++col) acc = fmaf(sm[tj][col], sx[tq][col], acc);
        __syncthreads();
    }
    const int j = j0 + tj, q = q0 + tq;
    if (j < r && q < k) part[((size_t)q * r + j) * nch + c] = (double)acc;
}

__global__ void k_coef_finish(const double *__restrict__ part, const double *__restrict__ w, double *__restrict__ C,
                              int r, int k, int nch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r * k) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(size_t)i * nch + c];
    C[i] = w ? s * w[i % r] : s;
}

// out[q][e] = base[q][e] + sign sum_j C[q][j] M[j][e]; each thread one e for
// kQ vectors; grid (points / 256, ceil(k / kQ)); C staged in shared memory.
constexpr int kQ = 16, kMaxR = 256;
__global__ void k_combine(const float *__restrict__ M, const double *__restrict__ C, const float *base, float sign,
                          float *out, int r, int k, size_t N)
{
    __shared__ float sc[kQ][kMaxR];
    const int q0 = blockIdx.y * kQ;
    for (int i = threadIdx.x; i < kQ * r; i += blockDim.x) {
        const int qq = i / r, j = i % r;
        sc[qq][j] = q0 + qq < k ? (float)C[(size_t)(q0 + qq) * r + j] : 0.0f;
    }
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    float acc[kQ];
#pragma unroll
    for (int qq = 0; qq < kQ; ++qq) acc[qq] = 0.0f;
    for (int j = 0; j < r; ++j) {
        const float m = M[(size_t)j * N + e];
#pragma unroll
        for (int qq = 0; qq < kQ; ++qq) acc[qq] = fmaf(sc[qq][j], m, acc[qq]);
    }
#pragma unroll
    for (int qq = 0; qq < kQ; ++qq) {
        const int q = q0 + qq;
        if (q < k) {
            const size_t t = (size_t)q * N + e;
            out[t] = (base ? base[t] : 0.0f) + sign * acc[qq];
        }
    }
}

}  // namespace

int chunks_of(size_t N) { return (int)((N + kChunk - 1) / kChunk); }

size_t rows_dot_scratch(int k, size_t N) { return (size_t)k * chunks_of(N); }

size_t coef_scratch(int r, int k, size_t N) { return (size_t)r * k * chunks_of(N); }

int rows_dot(const float *A, const float *B, double *out, int k, size_t N, double scale, double *scratch,
             cudaStream_t st)
{
    const int nch = chunks_of(N);
    k_rows_dot_part<<<dim3(nch, k), 256, 0, st>>>(A, B, scratch, N, nch);
    HV_RT_INTERNAL(launched("k_rows_dot_part"));
    k_sum_parts<<<nblk(k, 128), 128, 0, st>>>(scratch, out, k, nch, scale);
    return launched("k_sum_parts");
}

int coef(const float *M, int r, const float *X, int k, size_t N, const double *w, double *C, double *scratch,
         cudaStream_t st)
{
    const int nch = chunks_of(N);
    k_coef_part<<<dim3(nch, (r + kTile - 1) / kTile, (k + kTile - 1) / kTile), kTile * kTile, 0, st>>>(M, X, scratch,
                                                                                                     r, k, N, nch);
    HV_RT_INTERNAL(launched("k_coef_part"));
    k_coef_finish<<<nblk((size_t)r * k, 128), 128, 0, st>>>(scratch, w, C, r, k, nch);
    return launched("k_coef_finish");
}

int combine(const float *M, int r, const double *C, int k, size_t N, const float *base, float sign, float *out,
            cudaStream_t st)
{
    if (r > kMaxR) return hvi::fail(HV_EINVAL, "combine: %d terms (at most %d)", r, kMaxR);
    k_combine<<<dim3(nblk(N, 256), (k + kQ - 1) / kQ), 256, 0, st>>>(M, C, base, sign, out, r, k, N);
    return launched("k_combine");
}

}  // namespace hvk
