// hv_lowrank.cu -- the Matern prior operator and the low-rank (LR) Hessian
// approximation (sections 2.1 and 3.1).
//
// Prior: R = A^2, A = delta I - gamma Lap_h, Lap_h the 5-point Laplacian with
// homogeneous Neumann conditions (mirror ghost cells).  A is a stencil kernel;
// A^-1 = C^T diag(1 / (delta + gamma lambda)) C with C the orthonormal 2D
// DCT-II: in FP32 (the applies) by the fast transform of hv_dct.cu; in the FP64
// low-rank build as dense DGEMMs (Cz V Cx^T and back) on the cuBLAS library.
//
// LR: the r leading eigenpairs of H_d v = lambda R v by the randomized
// double-pass method with a caller-drawn Gaussian test matrix Omega:
//   Y = R^-1 H_d Omega, Q = R-orthonormalised Y (eigen-decomposition of the
//   R-Gram matrix in FP64, dropping directions below 1e-12 of the largest;
//   twice), T = Q^T H_d Q, T = S Lambda S^T, V = Q S[:, :r].
// Applies: H~_d v = R V Lambda V^T R v, and the sampling factor
// (I - V S_r V^T R) A^-1 with S_r = I - (Lambda + I)^-1/2, which maps N(0, I)
// to N(0, (H~_d + R)^-1).
// A product with R = A^2 amplifies the rounding of an R^-1-smoothed vector by
// up to cond(R) = cond(A)^2, so the build runs in FP64 (DGEMM transforms, FP64
// orthonormalisation; only the Hessian products are FP32) and keeps the
// factors V, W = A V and U = R V: the applies are U Lambda U^T v and
// A^-1 v - V S_r W^T v (V^T R A^-1 v = W^T v), with no product with R.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

namespace hvk {

namespace {

unsigned nb(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

int blas(cublasStatus_t s, const char *what)
{
    if (s != CUBLAS_STATUS_SUCCESS) return hvi::fail(HV_ECUDA, "%s: cuBLAS status %d", what, (int)s);
    return HV_OK;
}

// out = delta v - gamma Lap_h v for k fields [nz][nx] (mirror ghost cells);
// grid (columns / 128, nz, k).
template <class T>
__global__ void k_prior_A(const T *__restrict__ v, T *__restrict__ out, int nz, int nx, int k, T delta, T g_h2)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y;
    if (x >= nx) return;
    const size_t base = (size_t)blockIdx.z * nz * nx, t = base + (size_t)z * nx + x;
    const T c = v[t];
    const T n_ = v[base + (size_t)max(z - 1, 0) * nx + x], s_ = v[base + (size_t)min(z + 1, nz - 1) * nx + x];
    const T w_ = v[base + (size_t)z * nx + max(x - 1, 0)], e_ = v[base + (size_t)z * nx + min(x + 1, nx - 1)];
    out[t] = delta * c - g_h2 * (((n_ + s_) + (w_ + e_)) - T(4) * c);
}

// X[q][e] *= s[e]; grid (points / 256, k).
template <class T>
__global__ void k_scale_rows(T *__restrict__ X, const T *__restrict__ s, size_t N, int k)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N) X[(size_t)blockIdx.y * N + e] *= s[e];
}

template <class A, class B>
__global__ void k_convert(const A *__restrict__ in, B *__restrict__ out, size_t n)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (B)in[t];
}

// G[i][j] = sum_e X[i][e] Y[j][e] in FP64; one CTA per (i, j).
template <class TX, class TY>
__global__ void k_gram_real(const TX *__restrict__ X, const TY *__restrict__ Y, double *__restrict__ G, int kb,
                            size_t N)
{
    const int i = blockIdx.x, j = blockIdx.y;
    const TX *a = X + (size_t)i * N;
    const TY *b = Y + (size_t)j * N;
    double s = 0.0;
    for (size_t e = threadIdx.x; e < N; e += blockDim.x) s = fma((double)a[e], (double)b[e], s);
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[(size_t)i * kb + j] = sh[0];
}

// out[j][e] = sum_i M[i][j] X[i][e] (M: ki x ko, FP64).
__global__ void k_combine(const double *__restrict__ M, const double *__restrict__ X, double *__restrict__ out, int ki,
                          int ko, size_t N)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)ko * N) return;
    const int j = (int)(t / N);
    const size_t e = t - (size_t)j * N;
    double s = 0.0;
    for (int i = 0; i < ki; ++i) s = fma(M[(size_t)i * ko + j], X[(size_t)i * N + e], s);
    out[t] = s;
}

}  // namespace

// ------------------------------------------------------------------ prior
int prior_create(Prior &P, int nz, int nx, double h, double delta, double gamma)
{
    if (nz < 1 || nx < 1 || !(h > 0) || !(delta > 0) || !(gamma >= 0))
        return hvi::fail(HV_EINVAL, "prior: need nz, nx >= 1, h > 0, delta > 0, gamma >= 0");
    P.nz = nz;
    P.nx = nx;
    P.h = h;
    P.delta = delta;
    P.gamma = gamma;
    auto dct = [](int n) {
        std::vector<double> C((size_t)n * n);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                C[(size_t)k * n + j] = (k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n)) *
                                       std::cos(M_PI * k * (2.0 * j + 1.0) / (2.0 * n));
        return C;
    };
    const std::vector<double> Cz = dct(nz), Cx = dct(nx);
    std::vector<double> inv((size_t)nz * nx);
    for (int k = 0; k < nz; ++k)
        for (int l = 0; l < nx; ++l) {
            const double sz = std::sin(M_PI * k / (2.0 * nz)), sx = std::sin(M_PI * l / (2.0 * nx));
            inv[(size_t)k * nx + l] = 1.0 / (delta + gamma * (4.0 / (h * h)) * (sz * sz + sx * sx));
        }
    auto up = [&](const std::vector<double> &src, float **f, double **d) -> int {
        std::vector<float> sf(src.begin(), src.end());
        cudaError_t e;
        if ((e = cudaMalloc(f, sf.size() * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(d, src.size() * sizeof(double))) != cudaSuccess ||
            (e = cudaMemcpy(*f, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(*d, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return hvi::fail(HV_ECUDA, "prior tables: %s", cudaGetErrorString(e));
        return HV_OK;
    };
    HV_RT_INTERNAL(up(Cz, &P.Cz, &P.Czd));
    HV_RT_INTERNAL(up(Cx, &P.Cx, &P.Cxd));
    HV_RT_INTERNAL(up(inv, &P.inv, &P.invd));
    HV_RT_INTERNAL(blas(cublasCreate(&P.blas), "cublasCreate"));
    P.blas_ok = true;
    HV_RT_INTERNAL(blas(cublasSetMathMode(P.blas, CUBLAS_PEDANTIC_MATH), "cublasSetMathMode"));   // plain FP32/FP64
    return HV_OK;
}

void prior_destroy(Prior &P)
{
    dct_destroy(P.dct);
    if (P.blas_ok) cublasDestroy(P.blas);
    cudaFree(P.Cz);
    cudaFree(P.Cx);
    cudaFree(P.inv);
    cudaFree(P.Czd);
    cudaFree(P.Cxd);
    cudaFree(P.invd);
    cudaFree(P.tmp);
    cudaFree(P.tmpd);
    P = Prior{};
}

namespace {

template <class T>
int prior_tmp(Prior &P, int k, T **buf)
{
    void **slot = std::is_same<T, double>::value ? reinterpret_cast<void **>(&P.tmpd) : reinterpret_cast<void **>(&P.tmp);
    int &have = std::is_same<T, double>::value ? P.tmpd_k : P.tmp_k;
    if (have < k) {
        cudaFree(*slot);   // synchronises: nothing in flight uses the old scratch afterwards
        *slot = nullptr;
        have = 0;
        cudaError_t e = cudaMalloc(slot, (size_t)2 * k * P.nz * P.nx * sizeof(T));
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "prior scratch: %s", cudaGetErrorString(e));
        have = k;
    }
    *buf = reinterpret_cast<T *>(*slot);
    return HV_OK;
}

}  // namespace

// The FP32 A^-1 transform for batches of min(k, 64) fields (created once, or
// again for a larger batch while below 64).
constexpr int kDctBatch = 64;
int prior_dct(Prior &P, int k)
{
    const int want = std::min(std::max(k, 1), kDctBatch);
    if (P.dct.kmax >= want) return HV_OK;
    cudaDeviceSynchronize();   // nothing in flight uses the old transform afterwards
    dct_destroy(P.dct);
    return dct_create(P.dct, P.nz, P.nx, P.h, P.delta, P.gamma, want);
}

// Sizes the prior's FP32 scratch and transform for k fields now, so that later
// applies with at most k fields allocate nothing.
int prior_reserve(Prior &P, int k)
{
    float *buf = nullptr;
    HV_RT_INTERNAL(prior_tmp<float>(P, k, &buf));
    return prior_dct(P, k);
}

namespace {

// C = op(A) op(B), column-major, k-batched with the given strides.
int gemm_batched(cublasHandle_t hb, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int kk, const float *A,
                 int lda, long long sa, const float *B, int ldb, long long sb, float *C, int ldc, long long sc, int batch)
{
    const float one = 1.0f, zero = 0.0f;
    return blas(cublasSgemmStridedBatched(hb, ta, tb, m, n, kk, &one, A, lda, sa, B, ldb, sb, &zero, C, ldc, sc, batch),
                "cublasSgemmStridedBatched");
}
int gemm_batched(cublasHandle_t hb, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int kk, const double *A,
                 int lda, long long sa, const double *B, int ldb, long long sb, double *C, int ldc, long long sc, int batch)
{
    const double one = 1.0, zero = 0.0;
    return blas(cublasDgemmStridedBatched(hb, ta, tb, m, n, kk, &one, A, lda, sa, B, ldb, sb, &zero, C, ldc, sc, batch),
                "cublasDgemmStridedBatched");
}

template <class T>
int prior_A_t(const Prior &P, const T *v, T *out, int k, cudaStream_t st)
{
    k_prior_A<T><<<dim3(nb((size_t)P.nx, 128), P.nz, k), 128, 0, st>>>(v, out, P.nz, P.nx, k, (T)P.delta,
                                                                   (T)(P.gamma / (P.h * P.h)));
    return launched("k_prior_A");
}

// out = A^-1 v (k fields; out may equal v): the 2D DCT-II Cz V Cx^T, the
// eigenvalue scaling, and back (row-major fields seen as column-major).
template <class T>
int prior_Ainv_t(Prior &P, const T *Cz, const T *Cx, const T *inv, const T *v, T *out, int k, cudaStream_t st)
{
    const int nz = P.nz, nx = P.nx;
    const long long N = (long long)nz * nx;
    T *U = nullptr;
    HV_RT_INTERNAL(prior_tmp<T>(P, k, &U));
    T *Tm = U + (size_t)k * N;
    HV_RT_INTERNAL(blas(cublasSetStream(P.blas, st), "cublasSetStream"));
    HV_RT_INTERNAL(gemm_batched(P.blas, CUBLAS_OP_T, CUBLAS_OP_N, nx, nz, nx, Cx, nx, 0, v, nx, N, U, nx, N, k));
    HV_RT_INTERNAL(gemm_batched(P.blas, CUBLAS_OP_N, CUBLAS_OP_N, nx, nz, nz, U, nx, N, Cz, nz, 0, Tm, nx, N, k));
    k_scale_rows<T><<<dim3(nb((size_t)N, 256), k), 256, 0, st>>>(Tm, inv, (size_t)N, k);
    HV_RT_INTERNAL(launched("k_scale_rows"));
    HV_RT_INTERNAL(gemm_batched(P.blas, CUBLAS_OP_N, CUBLAS_OP_N, nx, nz, nx, Cx, nx, 0, Tm, nx, N, U, nx, N, k));
    HV_RT_INTERNAL(gemm_batched(P.blas, CUBLAS_OP_N, CUBLAS_OP_T, nx, nz, nz, U, nx, N, Cz, nz, 0, out, nx, N, k));
    return HV_OK;
}

}  // namespace

int prior_A(const Prior &P, const float *v, float *out, int k, cudaStream_t st) { return prior_A_t(P, v, out, k, st); }

int prior_Ainv(Prior &P, const float *v, float *out, int k, cudaStream_t st)
{
    HV_RT_INTERNAL(prior_dct(P, k));
    return dct_apply(P.dct, v, k, out, st);
}

int prior_R(Prior &P, const float *v, float *out, int k, cudaStream_t st)
{
    float *t = nullptr;
    HV_RT_INTERNAL(prior_tmp<float>(P, k, &t));
    HV_RT_INTERNAL(prior_A(P, v, t, k, st));
    return prior_A(P, t, out, k, st);
}

int prior_Rinv(Prior &P, const float *v, float *out, int k, cudaStream_t st)
{
    HV_RT_INTERNAL(prior_Ainv(P, v, out, k, st));
    return prior_Ainv(P, out, out, k, st);
}

// ------------------------------------------------------------------ LR
namespace {

struct DevBufs {   // device scratch freed on every exit path
    std::vector<void *> p;
    template <class T>
    int get(T **out, size_t n)
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(out), n * sizeof(T));
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "low-rank scratch: %s", cudaGetErrorString(e));
        p.push_back(*out);
        return HV_OK;
    }
    ~DevBufs()
    {
        for (void *q : p) cudaFree(q);
    }
};

int to_host(std::vector<double> &h, const double *d, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "low-rank build: %s", cudaGetErrorString(e));
    return HV_OK;
}

// Q (kk x N, FP64) <- an R-orthonormal basis of its span, through the
// eigen-decomposition of G = (A Q)^T (A Q); directions below 1e-12 of the
// largest eigenvalue are dropped; twice.  AQ, out: kk x N scratch.
int r_orthonormalise(Prior &P, double *Q, double *AQ, double *out, double *G, double *M, int k, size_t N, int *kout,
                     cudaStream_t st)
{
    int kk = k;
    for (int pass = 0; pass < 2; ++pass) {
        HV_RT_INTERNAL(prior_A_t(P, (const double *)Q, AQ, kk, st));
        k_gram_real<double, double><<<dim3(kk, kk), 256, 0, st>>>(AQ, AQ, G, kk, N);
        HV_RT_INTERNAL(launched("k_gram_real"));
        std::vector<double> Gh((size_t)kk * kk);
        HV_RT_INTERNAL(to_host(Gh, G, st));
        std::vector<std::complex<double>> Gc((size_t)kk * kk), U;
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < kk; ++j) Gc[(size_t)i * kk + j] = 0.5 * (Gh[(size_t)i * kk + j] + Gh[(size_t)j * kk + i]);
        std::vector<double> w;
        HV_RT_INTERNAL(hvi::hermitian_eig(kk, Gc, w, U));
        int keep = 0;
        while (keep < kk && w[keep] > 1e-12 * w[0]) ++keep;
        if (keep == 0) return hvi::fail(HV_EINVAL, "low-rank build: the test vectors span nothing");
        std::vector<double> Mh((size_t)kk * keep);
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < keep; ++j) Mh[(size_t)i * keep + j] = U[(size_t)i * kk + j].real() / std::sqrt(w[j]);
        cudaError_t e = cudaMemcpyAsync(M, Mh.data(), Mh.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "orthonormalisation: %s", cudaGetErrorString(e));
        k_combine<<<nb((size_t)keep * N, 256), 256, 0, st>>>(M, Q, out, kk, keep, N);
        HV_RT_INTERNAL(launched("k_combine"));
        e = cudaMemcpyAsync(Q, out, (size_t)keep * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // Mh is a host buffer of this pass
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "orthonormalisation: %s", cudaGetErrorString(e));
        kk = keep;
    }
    *kout = kk;
    return HV_OK;
}

}  // namespace

int build_lowrank(LowRank &L, const float *Y_in, int k, int rank, size_t N,
                  const std::function<int(const float *, int, float *)> &hessian, cudaStream_t st)
{
    // The build runs in FP64 (products with R of R^-1-smoothed vectors amplify rounding by cond(R));
    // H_d takes and returns FP32 fields.
    Prior &P = L.prior;
    DevBufs b;
    double *Q = nullptr, *AQ = nullptr, *X = nullptr, *G = nullptr, *M = nullptr;
    float *Q32 = nullptr, *Z32 = nullptr;
    HV_RT_INTERNAL(b.get(&Q, (size_t)k * N));
    HV_RT_INTERNAL(b.get(&AQ, (size_t)k * N));
    HV_RT_INTERNAL(b.get(&X, (size_t)k * N));
    HV_RT_INTERNAL(b.get(&G, (size_t)k * k));
    HV_RT_INTERNAL(b.get(&M, (size_t)k * k));
    HV_RT_INTERNAL(b.get(&Q32, (size_t)k * N));
    HV_RT_INTERNAL(b.get(&Z32, (size_t)k * N));
    // Y = R^-1 H_d Omega (FP64)
    k_convert<float, double><<<nb((size_t)k * N, 256), 256, 0, st>>>(Y_in, Q, (size_t)k * N);
    HV_RT_INTERNAL(launched("k_convert"));
    HV_RT_INTERNAL(prior_Ainv_t(P, P.Czd, P.Cxd, P.invd, (const double *)Q, Q, k, st));
    HV_RT_INTERNAL(prior_Ainv_t(P, P.Czd, P.Cxd, P.invd, (const double *)Q, Q, k, st));
    int kk = k;
    HV_RT_INTERNAL(r_orthonormalise(P, Q, AQ, X, G, M, k, N, &kk, st));
    if (rank > kk) return hvi::fail(HV_EINVAL, "the test vectors span %d directions; rank %d asked", kk, rank);
    // second pass: T = Q^T H_d Q
    k_convert<double, float><<<nb((size_t)kk * N, 256), 256, 0, st>>>(Q, Q32, (size_t)kk * N);
    HV_RT_INTERNAL(launched("k_convert"));
    HV_RT_INTERNAL(hessian(Q32, kk, Z32));
    k_gram_real<double, float><<<dim3(kk, kk), 256, 0, st>>>(Q, Z32, G, kk, N);
    HV_RT_INTERNAL(launched("k_gram_real"));
    std::vector<double> Th((size_t)kk * kk);
    HV_RT_INTERNAL(to_host(Th, G, st));
    std::vector<std::complex<double>> Tc((size_t)kk * kk), S;
    for (int i = 0; i < kk; ++i)
        for (int j = 0; j < kk; ++j) Tc[(size_t)i * kk + j] = 0.5 * (Th[(size_t)i * kk + j] + Th[(size_t)j * kk + i]);
    std::vector<double> lam;
    HV_RT_INTERNAL(hvi::hermitian_eig(kk, Tc, lam, S));
    L.r = rank;
    L.N = N;
    L.mu = new std::mutex;
    L.lam.assign(lam.begin(), lam.begin() + rank);
    std::vector<double> Sh((size_t)kk * rank), wh(2 * (size_t)rank);
    for (int i = 0; i < kk; ++i)
        for (int j = 0; j < rank; ++j) Sh[(size_t)i * rank + j] = S[(size_t)i * kk + j].real();
    for (int j = 0; j < rank; ++j) {
        wh[j] = L.lam[j];                                        // H: Lambda
        wh[rank + j] = 1.0 - 1.0 / std::sqrt(L.lam[j] + 1.0);   // sampling: S_r
    }
    cudaError_t e;
    if ((e = cudaMalloc(&L.V, (size_t)rank * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&L.W, (size_t)rank * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&L.U, (size_t)rank * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&L.w, wh.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.w, wh.data(), wh.size() * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(M, Sh.data(), Sh.size() * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "low-rank factors: %s", cudaGetErrorString(e));
    // V = Q S[:, :r], W = A V, U = A W = R V (FP64), stored in FP32
    k_combine<<<nb((size_t)rank * N, 256), 256, 0, st>>>(M, Q, X, kk, rank, N);
    HV_RT_INTERNAL(launched("k_combine"));
    HV_RT_INTERNAL(prior_A_t(P, (const double *)X, AQ, rank, st));
    HV_RT_INTERNAL(prior_A_t(P, (const double *)AQ, Q, rank, st));
    const size_t n = (size_t)rank * N;
    k_convert<double, float><<<nb(n, 256), 256, 0, st>>>(X, L.V, n);
    k_convert<double, float><<<nb(n, 256), 256, 0, st>>>(AQ, L.W, n);
    k_convert<double, float><<<nb(n, 256), 256, 0, st>>>(Q, L.U, n);
    HV_RT_INTERNAL(launched("k_convert"));
    e = cudaStreamSynchronize(st);   // the scratch is freed on return
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "low-rank build: %s", cudaGetErrorString(e));
    return HV_OK;
}

void lowrank_destroy(LowRank &L)
{
    prior_destroy(L.prior);
    cudaFree(L.V);
    cudaFree(L.W);
    cudaFree(L.U);
    cudaFree(L.w);
    cudaFree(L.c);
    cudaFree(L.x);
    cudaFree(L.red);
    if (L.done) cudaEventDestroy(L.done);
    delete L.mu;
    L = LowRank{};
}

// mode 0: out = U Lambda U^T v (U = R V: R V Lambda V^T R v); mode 2: out = A^-1 v - V S_r W^T v.
// k vectors at once: the coefficient and combination products of hv_blas.cu.
int lowrank_apply(LowRank &L, const float *v, int k, float *out, int mode, cudaStream_t st)
{
    const size_t N = L.N;
    std::lock_guard<std::mutex> lk(*L.mu);
    cudaError_t e = cudaStreamWaitEvent(st, L.done, 0);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
    if (L.xk < k) {
        cudaFree(L.x);   // synchronises: nothing in flight uses the old scratch afterwards
        cudaFree(L.c);
        cudaFree(L.red);
        L.x = nullptr;
        L.c = nullptr;
        L.red = nullptr;
        L.xk = 0;
        if ((e = cudaMalloc(&L.x, (size_t)k * N * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&L.c, (size_t)k * L.r * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&L.red, coef_scratch(L.r, k, N) * sizeof(double))) != cudaSuccess)
            return hvi::fail(HV_ECUDA, "low-rank apply scratch: %s", cudaGetErrorString(e));
        L.xk = k;
    }
    if (mode == 0) {
        HV_RT_INTERNAL(coef(L.U, L.r, v, k, N, L.w, L.c, L.red, st));
        HV_RT_INTERNAL(combine(L.U, L.r, L.c, k, N, nullptr, 1.0f, out, st));
    } else {
        HV_RT_INTERNAL(prior_Ainv(L.prior, v, L.x, k, st));
        HV_RT_INTERNAL(coef(L.W, L.r, v, k, N, L.w + L.r, L.c, L.red, st));
        HV_RT_INTERNAL(combine(L.V, L.r, L.c, k, N, L.x, -1.0f, out, st));
    }
    e = cudaEventRecord(L.done, st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    return HV_OK;
}

}  // namespace hvk
