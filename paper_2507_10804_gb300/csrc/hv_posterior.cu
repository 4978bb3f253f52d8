// hv_posterior.cu -- the Laplace approximation of the posterior built from a
// Hessian approximation (sections 2.2, 3.1, 3.7) and the gpCN step (section 2.3).
//
// H0 = H~_d + R with R = A^2 the Matern prior and H~_d = B B^T a square-root
// (SPD) low-rank-symbol approximation, or H~_d = 0.  Solves with H0 (and with
// Op + R for a caller's operator) run preconditioned conjugate gradients,
// preconditioner R^-1, k right-hand sides at once: FP32 vectors, FP64 dot
// products and step lengths.  Posterior samples: y = A n1 + B n2 ~ N(0, H0),
// z = H0^-1 y ~ N(0, H0^-1) (for H~_d = 0, z = A^-1 n1 exactly).
//
// Low-rank correction: the leading eigenpairs of (H_d - H~_d) v = lambda H0 v,
// V^T H0 V = I, by the randomized double pass with H0 in place of R:
//   Z = (H_d - H~_d) Omega, Y = H0^-1 Z (so H0 Y = Z), Q = Y M with M from the
//   eigen-decomposition of the H0-Gram matrix Y^T Z (FP64; directions below
//   1e-12 of the largest dropped; twice, carrying H0 Q = Z M along), T = Q^T
//   (H_d - H~_d) Q = S Lambda S^T, V = Q S[:, :r], U = H0 V = (H0 Q) S[:, :r].
// Then H~ = H0 + U Lambda U^T and zeta = z - V S_r U^T z, S_r = I - (Lambda + I)^-1/2,
// z ~ N(0, H0^-1), is a sample of N(0, H~^-1).  Carrying H0 Q avoids every
// product of H0 with an H0^-1-smoothed vector (which would amplify the FP32
// rounding by cond(H0)).
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <mutex>
#include <vector>

#define PCK(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Scratch of the solves, applies and the correction, allocated once at
// hv_posterior_create for at most k = max_k fields: 7 k-field buffers (CG r,
// z, p, q, R p, and two for the sampler), 5 k-vectors of FP64 CG scalars,
// k x 256 correction coefficients, k activity flags; for the correction 6
// k-field buffers and two k x k FP64 matrices.
struct PostWork {
    int k = 0;
    float *f = nullptr;
    double *d = nullptr;
    double *red = nullptr;   // reduction partials (hv_blas.cu)
    int *act = nullptr;
    float *cf = nullptr;     // correction fields [6][k][N]
    double *cm = nullptr;    // correction matrices [2][k][k]
};

struct hv_posterior {
    int device = -1;
    int nz = 0, nx = 0;
    double h = 0;
    hvk::Prior prior;
    const hv_approx *approx = nullptr;    // borrowed square-root approximation, or null
    int r = 0;                            // correction rank
    std::vector<double> lam;
    float *V = nullptr, *U = nullptr;     // [r][N] (room for max_k rows)
    double *w = nullptr;                  // [2r]: Lambda, S_r (room for 2 max_k)
    PostWork work;
    cudaEvent_t done = nullptr;           // last use of the scratch and the prior's tables
    std::mutex *mu = nullptr;
};

namespace {

using OpFn = std::function<int(const float *, int, float *)>;

unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched(const char *what)
{
    hvk::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

// Build-time products of the correction (FP64 accumulation throughout: the
// orthonormalisation combines nearly dependent vectors with large weights).
// G[i][j] = sum_e X[i][e] Y[j][e]; one CTA per (i, j).
__global__ void k_gram_rows(const float *__restrict__ X, const float *__restrict__ Y, double *__restrict__ G, int kb,
                            size_t N)
{
    const int i = blockIdx.x, j = blockIdx.y;
    const float *a = X + (size_t)i * N, *b = Y + (size_t)j * N;
    double acc = 0.0;
    for (size_t e = threadIdx.x; e < N; e += blockDim.x) acc = fma((double)a[e], (double)b[e], acc);
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[(size_t)i * kb + j] = sh[0];
}

// out[j][e] = sum_i M[i][j] X[i][e] (M: ki x ko).
__global__ void k_combine_rows(const double *__restrict__ M, const float *__restrict__ X, float *__restrict__ out,
                               int ki, int ko, size_t N)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)ko * N) return;
    const int j = (int)(t / N);
    const size_t e = t - (size_t)j * N;
    double s = 0.0;
    for (int i = 0; i < ki; ++i) s = fma(M[(size_t)i * ko + j], (double)X[(size_t)i * N + e], s);
    out[t] = (float)s;
}

// out = a + s b  (out may be a).
__global__ void k_axpy(const float *a, const float *__restrict__ b, float s, float *out, size_t n)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = fmaf(s, b[t], a[t]);
}

// CG step lengths (FP64 quotients, once per vector): alpha[q] = active ? rz[q] / pq[q] : 0.
__global__ void k_cg_alpha(const double *__restrict__ rz, const double *__restrict__ pq, const int *__restrict__ act,
                           double *__restrict__ alpha, int k)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < k) alpha[q] = (act[q] && pq[q] > 0.0) ? rz[q] / pq[q] : 0.0;
}

// beta[q] = active ? rz_new[q] / rz[q] : 0, then rz <- rz_new.
__global__ void k_cg_beta(const double *__restrict__ rz_new, double *__restrict__ rz, const int *__restrict__ act,
                          double *__restrict__ beta, int k)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    beta[q] = (act[q] && rz[q] > 0.0) ? rz_new[q] / rz[q] : 0.0;
    rz[q] = rz_new[q];
}

// x += alpha p, r -= alpha q (per vector); grid (points / 256, k).
__global__ void k_cg_xr(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
                        const float *__restrict__ q, const double *__restrict__ alpha, int k, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const size_t t = (size_t)blockIdx.y * N + e;
    const float a = (float)alpha[blockIdx.y];   // FP32 updates: the vectors are FP32
    x[t] = fmaf(a, p[t], x[t]);
    r[t] = fmaf(-a, q[t], r[t]);
}

// p = z + beta p (beta from k_cg_beta); grid (points / 256, k).
__global__ void k_cg_p(float *__restrict__ p, const float *__restrict__ z, const double *__restrict__ beta, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const size_t t = (size_t)blockIdx.y * N + e;
    p[t] = fmaf((float)beta[blockIdx.y], p[t], z[t]);
}

// gpCN proposal: m' = map + sqrt(1 - beta^2)(m - map) + beta zeta, d = m' - map;
// grid (points / 256, c).
__global__ void k_gpcn_propose(const float *__restrict__ m, const float *__restrict__ map,
                               const float *__restrict__ zeta, float s, float beta, float *__restrict__ mp,
                               float *__restrict__ d, int c, size_t N)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const size_t t = (size_t)blockIdx.y * N + e;
    const float m0 = map[e];
    const float dd = fmaf(s, m[t] - m0, beta * zeta[t]);
    mp[t] = m0 + dd;
    if (d) d[t] = dd;
}

// gpCN acceptance, one CTA of 256 threads per chain: the dot dHd = d . Hd of
// the chain's n values (double-float accumulation on the FP32 pipe inside a
// thread -- each product split exactly, about 2^-44 relative -- then an FP64
// tree over the threads, a fixed order), Delta' = phi' - 1/2 dHd, and the
// decision: accept iff log_u < Delta_cur - Delta'; on acceptance Delta_cur <- Delta'.
__global__ void __launch_bounds__(256) k_gpcn_decide(const double *__restrict__ phi_new, const float *__restrict__ d,
                                                     const float *__restrict__ Hd, const double *__restrict__ log_u,
                                                     double *__restrict__ delta_cur, int *__restrict__ accepted,
                                                     size_t n)
{
    __shared__ double sh[256];
    const int c = blockIdx.x;
    const float *a = d + (size_t)c * n, *b = Hd + (size_t)c * n;
    float hi = 0.0f, lo = 0.0f;
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
        const float x = a[e], y = b[e];
        const float p = __fmul_rn(x, y), pe = fmaf(x, y, -p);
        const float s = __fadd_rn(hi, p), bv = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv)), pe));
        hi = s;
    }
    sh[threadIdx.x] = (double)hi + (double)lo;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dn = phi_new[c] - 0.5 * sh[0];
        const int take = log_u[c] < delta_cur[c] - dn;
        if (take) delta_cur[c] = dn;
        accepted[c] = take;
    }
}

// m[c] <- m_new[c] for the accepted chains; grid (points / 256, c).
__global__ void k_gpcn_take(const float *__restrict__ mp, const int *__restrict__ accepted, float *__restrict__ m,
                            size_t N)
{
    const int c = blockIdx.y;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N && accepted[c]) m[(size_t)c * N + e] = mp[(size_t)c * N + e];
}

constexpr int kWorkFields = 7, kMaxCorrection = 256;

// Holds the posterior's lock and orders `st` after the previous user of its
// scratch (which may have run on another stream); records the next use on exit.
struct Session {
    std::lock_guard<std::mutex> lk;
    hv_posterior *p;
    cudaStream_t st;
    Session(hv_posterior *p_, cudaStream_t st_) : lk(*p_->mu), p(p_), st(st_) { cudaStreamWaitEvent(st, p->done, 0); }
    ~Session() { cudaEventRecord(p->done, st); }
};

// Allocates the scratch for up to k fields (at create only).
int alloc_work(PostWork &w, int k, size_t N)
{
    cudaError_t e;
    if ((e = cudaMalloc(&w.f, (size_t)kWorkFields * k * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w.d, (size_t)(5 + kMaxCorrection) * k * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&w.red, hvk::coef_scratch(kMaxCorrection, k, N) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&w.act, (size_t)k * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&w.cf, (size_t)6 * k * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w.cm, (size_t)2 * k * k * sizeof(double))) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "posterior scratch: %s", cudaGetErrorString(e));
    w.k = k;
    return HV_OK;
}

// Calls take at most the k fields the scratch was sized for.
int check_k(const PostWork &w, int k)
{
    if (k > w.k) return hvi::fail(HV_EINVAL, "k = %d fields; this posterior was created for at most %d", k, w.k);
    return HV_OK;
}

// Field buffer i (0..6) of the cached scratch, sized for k fields.
float *work_field(const PostWork &w, int i, size_t N) { return w.f + (size_t)i * w.k * N; }

int check_device(int device)
{
    int dev = -1;
    PCK(cudaGetDevice(&dev));
    if (dev != device) return hvi::fail(HV_EINVAL, "current device %d is not the object's device %d", dev, device);
    return HV_OK;
}

// out = (Op + R) v for k fields; Op may be empty (out = R v).  t: k-field scratch.
int apply_op_plus_R(hvk::Prior &P, const OpFn &op, const float *v, int k, float *out, float *t, cudaStream_t st)
{
    const size_t n = (size_t)k * P.nz * P.nx;
    if (!op) return hvk::prior_R(P, v, out, k, st);
    HV_RT_INTERNAL(op(v, k, out));
    HV_RT_INTERNAL(hvk::prior_R(P, v, t, k, st));
    k_axpy<<<nblk(n, 256), 256, 0, st>>>(out, t, 1.0f, out, n);
    return launched("k_axpy");
}

// Preconditioned CG for (Op + R) X = B, k right-hand sides, preconditioner R^-1.
// Uses fields 0..4 and the scalars of the cached scratch w (sized for >= k).
int pcg(hvk::Prior &P, const OpFn &op, const float *b, int k, float *x, double rtol, int max_iter, int *iters,
        cudaStream_t st, const PostWork &w)
{
    const size_t N = (size_t)P.nz * P.nx, n = (size_t)k * N;
    float *r = work_field(w, 0, N), *z = work_field(w, 1, N), *p = work_field(w, 2, N), *q = work_field(w, 3, N),
          *t = work_field(w, 4, N);
    double *rz = w.d, *rz_new = w.d + w.k, *pq = w.d + 2 * w.k, *alpha = w.d + 3 * w.k, *rr = w.d + 4 * w.k;
    int *act = w.act;
    PCK(cudaMemsetAsync(x, 0, n * sizeof(float), st));
    PCK(cudaMemcpyAsync(r, b, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    HV_RT_INTERNAL(hvk::rows_dot(b, b, rr, k, N, 1.0, w.red, st));
    std::vector<double> bb(k), rh(k);
    std::vector<int> ah(k);
    PCK(cudaMemcpyAsync(bb.data(), rr, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    int live = 0;
    for (int j = 0; j < k; ++j) live += (ah[j] = bb[j] > 0.0);
    PCK(cudaMemcpyAsync(act, ah.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    HV_RT_INTERNAL(hvk::prior_Rinv(P, r, z, k, st));
    PCK(cudaMemcpyAsync(p, z, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    HV_RT_INTERNAL(hvk::rows_dot(r, z, rz, k, N, 1.0, w.red, st));
    int it = 0;
    while (live > 0) {
        if (it >= max_iter) {
            if (iters) *iters = it;
            return hvi::fail(HV_ETIMEOUT, "conjugate gradients: %d of %d vectors above rtol %g after %d iterations",
                             live, k, rtol, it);
        }
        ++it;
        HV_RT_INTERNAL(apply_op_plus_R(P, op, p, k, q, t, st));
        HV_RT_INTERNAL(hvk::rows_dot(p, q, pq, k, N, 1.0, w.red, st));
        k_cg_alpha<<<nblk(k, 128), 128, 0, st>>>(rz, pq, act, alpha, k);
        HV_RT_INTERNAL(launched("k_cg_alpha"));
        k_cg_xr<<<dim3(nblk(N, 256), k), 256, 0, st>>>(x, r, p, q, alpha, k, N);
        HV_RT_INTERNAL(launched("k_cg_xr"));
        HV_RT_INTERNAL(hvk::rows_dot(r, r, rr, k, N, 1.0, w.red, st));
        PCK(cudaMemcpyAsync(rh.data(), rr, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        PCK(cudaStreamSynchronize(st));
        live = 0;
        for (int j = 0; j < k; ++j) live += (ah[j] = ah[j] && rh[j] > rtol * rtol * bb[j]);
        if (live == 0) break;
        PCK(cudaMemcpyAsync(act, ah.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
        HV_RT_INTERNAL(hvk::prior_Rinv(P, r, z, k, st));
        HV_RT_INTERNAL(hvk::rows_dot(r, z, rz_new, k, N, 1.0, w.red, st));
        k_cg_beta<<<nblk(k, 128), 128, 0, st>>>(rz_new, rz, act, alpha, k);   // alpha's slot holds beta now
        HV_RT_INTERNAL(launched("k_cg_beta"));
        k_cg_p<<<dim3(nblk(N, 256), k), 256, 0, st>>>(p, z, alpha, N);
        HV_RT_INTERNAL(launched("k_cg_p"));
    }
    if (iters) *iters = it;
    return HV_OK;
}

OpFn gram_op(const hv_posterior *p, cudaStream_t st)
{
    if (!p->approx) return OpFn();
    hvk::LrSym *lr = const_cast<hvk::LrSym *>(&p->approx->lr);
    return [lr, st](const float *X, int k, float *Z) { return hvk::lr_apply(*lr, X, k, Z, st, hvk::kLrGram); };
}

OpFn user_op(const hv_operator *op, cudaStream_t st)
{
    return [op, st](const float *X, int k, float *Z) {
        const int rc = op->apply(op->ctx, X, k, Z, (void *)st);
        return rc == HV_OK ? HV_OK : hvi::fail(rc, "the operator's apply returned %d", rc);
    };
}

// Symmetric FP64 matrix [n][n] on the device -> eigenpairs on the host (descending).
int device_eig(const double *G, int n, std::vector<double> &w, std::vector<double> &Vr, cudaStream_t st)
{
    std::vector<double> Gh((size_t)n * n);
    PCK(cudaMemcpyAsync(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    std::vector<std::complex<double>> Gc((size_t)n * n), Vc;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Gc[(size_t)i * n + j] = 0.5 * (Gh[(size_t)i * n + j] + Gh[(size_t)j * n + i]);
    HV_RT_INTERNAL(hvi::hermitian_eig(n, Gc, w, Vc));
    Vr.resize((size_t)n * n);
    for (size_t i = 0; i < Vr.size(); ++i) Vr[i] = Vc[i].real();
    return HV_OK;
}

}  // namespace

extern "C" int hv_posterior_create(int nz, int nx, double h, double delta, double gamma, const hv_approx *approx,
                                   int max_k, hv_posterior **out)
{
    if (out) *out = nullptr;
    if (!out) return hvi::fail(HV_EINVAL, "null output");
    if (max_k < 1 || max_k > kMaxCorrection)
        return hvi::fail(HV_EINVAL, "max_k = %d; need 1 <= max_k <= %d", max_k, kMaxCorrection);
    if (approx) {
        if ((approx->kind != 1 && approx->kind != 2) || !approx->lr.spd)
            return hvi::fail(HV_EINVAL, "the posterior takes a square-root (SPD) PDO or PSF+ approximation");
        if (approx->lr.g.nz != nz || approx->lr.g.nx != nx)
            return hvi::fail(HV_EINVAL, "the approximation is on a %d x %d grid, not %d x %d", approx->lr.g.nz,
                             approx->lr.g.nx, nz, nx);
    }
    int dev = -1;
    PCK(cudaGetDevice(&dev));
    if (approx && approx->device != dev) return hvi::fail(HV_EINVAL, "the approximation is on device %d", approx->device);
    hv_posterior *p = new hv_posterior;
    p->device = dev;
    p->nz = nz;
    p->nx = nx;
    p->h = h;
    p->approx = approx;
    p->mu = new std::mutex;
    const size_t N = (size_t)nz * nx;
    int rc = hvk::prior_create(p->prior, nz, nx, h, delta, gamma);
    if (rc == HV_OK) rc = hvk::prior_reserve(p->prior, max_k);
    if (rc == HV_OK) rc = alloc_work(p->work, max_k, N);
    if (rc == HV_OK && (cudaMalloc(&p->V, (size_t)max_k * N * sizeof(float)) != cudaSuccess ||
                        cudaMalloc(&p->U, (size_t)max_k * N * sizeof(float)) != cudaSuccess ||
                        cudaMalloc(&p->w, (size_t)2 * max_k * sizeof(double)) != cudaSuccess))
        rc = hvi::fail(HV_ECUDA, "posterior correction factors: out of device memory");
    if (rc == HV_OK && cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess)
        rc = hvi::fail(HV_ECUDA, "cudaEventCreate failed");
    if (rc != HV_OK) {
        hv_posterior_destroy(p);
        return rc;
    }
    *out = p;
    return HV_OK;
}

extern "C" int hv_posterior_destroy(hv_posterior *p)
{
    if (!p) return HV_OK;
    cudaDeviceSynchronize();
    hvk::prior_destroy(p->prior);
    cudaFree(p->V);
    cudaFree(p->U);
    cudaFree(p->w);
    cudaFree(p->work.f);
    cudaFree(p->work.d);
    cudaFree(p->work.red);
    cudaFree(p->work.act);
    cudaFree(p->work.cf);
    cudaFree(p->work.cm);
    if (p->done) cudaEventDestroy(p->done);
    delete p->mu;
    delete p;
    return HV_OK;
}

extern "C" int hv_posterior_solve(hv_posterior *p, const hv_operator *op, const float *b, int k, float *x, double rtol,
                                  int max_iter, int *iters, void *stream)
{
    if (iters) *iters = 0;
    if (!p || !b || !x) return hvi::fail(HV_EINVAL, "null posterior, right-hand side or solution");
    if (k < 1 || k > 4096) return hvi::fail(HV_EINVAL, "k = %d; need 1 <= k <= 4096", k);
    if (!(rtol > 0 && rtol < 1) || max_iter < 1) return hvi::fail(HV_EINVAL, "rtol %g, max_iter %d", rtol, max_iter);
    if (op && (!op->apply || op->nz != p->nz || op->nx != p->nx))
        return hvi::fail(HV_EINVAL, "the operator does not act on the posterior's grid");
    HV_RT_INTERNAL(check_device(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    Session ses(p, st);
    HV_RT_INTERNAL(check_k(p->work, k));
    return pcg(p->prior, op ? user_op(op, st) : gram_op(p, st), b, k, x, rtol, max_iter, iters, st, p->work);
}

extern "C" int hv_posterior_apply(hv_posterior *p, const float *v, int k, float *out, void *stream)
{
    if (!p || !v || !out) return hvi::fail(HV_EINVAL, "null posterior, vector or output");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "k = %d; need 1 <= k <= 65535", k);
    HV_RT_INTERNAL(check_device(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    Session ses(p, st);
    const size_t N = (size_t)p->nz * p->nx;
    HV_RT_INTERNAL(check_k(p->work, k));
    float *t = work_field(p->work, 4, N);
    double *C = p->work.d + 5 * (size_t)p->work.k;
    HV_RT_INTERNAL(apply_op_plus_R(p->prior, gram_op(p, st), v, k, out, t, st));
    if (p->r > 0) {
        HV_RT_INTERNAL(hvk::coef(p->U, p->r, v, k, N, p->w, C, p->work.red, st));
        HV_RT_INTERNAL(hvk::combine(p->U, p->r, C, k, N, out, 1.0f, out, st));
    }
    return HV_OK;
}

extern "C" int hv_posterior_sample(hv_posterior *p, const float *n1, const float *n2, int k, float *zeta, double rtol,
                                   int max_iter, int *iters, void *stream)
{
    if (iters) *iters = 0;
    if (!p || !n1 || !zeta || (p->approx && !n2)) return hvi::fail(HV_EINVAL, "null posterior, normals or output");
    if (k < 1 || k > 4096) return hvi::fail(HV_EINVAL, "k = %d; need 1 <= k <= 4096", k);
    if (!(rtol > 0 && rtol < 1) || max_iter < 1) return hvi::fail(HV_EINVAL, "rtol %g, max_iter %d", rtol, max_iter);
    HV_RT_INTERNAL(check_device(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    Session ses(p, st);
    const size_t N = (size_t)p->nz * p->nx, n = (size_t)k * N;
    HV_RT_INTERNAL(check_k(p->work, k));
    if (!p->approx) {
        HV_RT_INTERNAL(hvk::prior_Ainv(p->prior, n1, zeta, k, st));   // H0^-1 A n1 = A^-1 n1
    } else {
        float *y = work_field(p->work, 5, N), *t = work_field(p->work, 6, N);
        HV_RT_INTERNAL(hvk::prior_A(p->prior, n1, y, k, st));
        HV_RT_INTERNAL(hvk::lr_apply(const_cast<hvk::LrSym &>(p->approx->lr), n2, k, t, st, hvk::kLrForward));
        k_axpy<<<nblk(n, 256), 256, 0, st>>>(y, t, 1.0f, y, n);
        HV_RT_INTERNAL(launched("k_axpy"));
        HV_RT_INTERNAL(pcg(p->prior, gram_op(p, st), y, k, zeta, rtol, max_iter, iters, st, p->work));
    }
    if (p->r > 0) {
        double *C = p->work.d + 5 * (size_t)p->work.k;
        HV_RT_INTERNAL(hvk::coef(p->U, p->r, zeta, k, N, p->w + p->r, C, p->work.red, st));
        HV_RT_INTERNAL(hvk::combine(p->V, p->r, C, k, N, zeta, -1.0f, zeta, st));
    }
    return HV_OK;
}

extern "C" int hv_posterior_correct(hv_posterior *p, const hv_operator *hd, const float *omega, int k, int rank,
                                    double rtol, int max_iter, void *stream)
{
    if (!p || !hd || !hd->apply || !omega) return hvi::fail(HV_EINVAL, "null posterior, operator or test vectors");
    if (hd->nz != p->nz || hd->nx != p->nx) return hvi::fail(HV_EINVAL, "the operator does not act on the posterior's grid");
    if (rank < 1 || k < rank || k > kMaxCorrection) return hvi::fail(HV_EINVAL, "rank %d with %d test vectors; need 1 <= rank <= k <= 256", rank, k);
    HV_RT_INTERNAL(check_k(p->work, k));
    if (!(rtol > 0 && rtol < 1) || max_iter < 1) return hvi::fail(HV_EINVAL, "rtol %g, max_iter %d", rtol, max_iter);
    HV_RT_INTERNAL(check_device(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    Session ses(p, st);
    const size_t N = (size_t)p->nz * p->nx, n = (size_t)k * N;
    // the correction's scratch, sized at create for max_k fields
    const size_t cap = (size_t)p->work.k * N;
    float *Z = p->work.cf, *Y = Z + cap, *HQ = Y + cap, *t = HQ + cap, *Q2 = t + cap, *HQ2 = Q2 + cap;
    double *G = p->work.cm, *M = G + (size_t)p->work.k * p->work.k;
    const OpFn H = user_op(hd, st), B = gram_op(p, st);
    auto resid = [&](const float *X, int kk, float *out) {   // (H_d - H~_d) X
        HV_RT_INTERNAL(H(X, kk, out));
        if (!B) return HV_OK;
        HV_RT_INTERNAL(B(X, kk, t));
        const size_t m = (size_t)kk * N;
        k_axpy<<<nblk(m, 256), 256, 0, st>>>(out, t, -1.0f, out, m);
        return launched("k_axpy");
    };
    // Z = (H_d - H~_d) Omega, Y = H0^-1 Z
    HV_RT_INTERNAL(resid(omega, k, Z));
    if (!p->approx) {
        HV_RT_INTERNAL(hvk::prior_Rinv(p->prior, Z, Y, k, st));
    } else {
        HV_RT_INTERNAL(pcg(p->prior, B, Z, k, Y, rtol, max_iter, nullptr, st, p->work));
    }
    // H0-orthonormalise Y, carrying H0 Y = Z along: Q <- Y, HQ <- Z
    PCK(cudaMemcpyAsync(HQ, Z, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    float *Q = Y;
    int kk = k;
    for (int pass = 0; pass < 2; ++pass) {
        k_gram_rows<<<dim3(kk, kk), 256, 0, st>>>(Q, HQ, G, kk, N);
        HV_RT_INTERNAL(launched("k_gram_rows"));
        std::vector<double> w, Uv;
        HV_RT_INTERNAL(device_eig(G, kk, w, Uv, st));
        int keep = 0;
        while (keep < kk && w[keep] > 1e-12 * w[0]) ++keep;
        if (keep == 0) return hvi::fail(HV_EINVAL, "correction: the test vectors span nothing");
        std::vector<double> Mh((size_t)kk * keep);
        for (int i = 0; i < kk; ++i)
            for (int j = 0; j < keep; ++j) Mh[(size_t)i * keep + j] = Uv[(size_t)i * kk + j] / std::sqrt(w[j]);
        PCK(cudaMemcpyAsync(M, Mh.data(), Mh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        k_combine_rows<<<nblk((size_t)keep * N, 256), 256, 0, st>>>(M, Q, Q2, kk, keep, N);
        HV_RT_INTERNAL(launched("k_combine_rows"));
        k_combine_rows<<<nblk((size_t)keep * N, 256), 256, 0, st>>>(M, HQ, HQ2, kk, keep, N);
        HV_RT_INTERNAL(launched("k_combine_rows"));
        PCK(cudaStreamSynchronize(st));   // Mh is this pass's host buffer
        std::swap(Q, Q2);
        std::swap(HQ, HQ2);
        kk = keep;
    }
    if (rank > kk) return hvi::fail(HV_EINVAL, "the test vectors span %d directions; rank %d asked", kk, rank);
    // T = Q^T (H_d - H~_d) Q
    HV_RT_INTERNAL(resid(Q, kk, Z));
    k_gram_rows<<<dim3(kk, kk), 256, 0, st>>>(Q, Z, G, kk, N);
    HV_RT_INTERNAL(launched("k_gram_rows"));
    std::vector<double> lam, S;
    HV_RT_INTERNAL(device_eig(G, kk, lam, S, st));
    for (int j = 0; j < rank; ++j)
        if (!(lam[j] > -1.0))
            return hvi::fail(HV_EINVAL, "correction eigenvalue %d is %g <= -1: H~ would not be positive definite", j, lam[j]);
    std::vector<double> Sh((size_t)kk * rank), wh(2 * (size_t)rank);
    for (int i = 0; i < kk; ++i)
        for (int j = 0; j < rank; ++j) Sh[(size_t)i * rank + j] = S[(size_t)i * kk + j];
    for (int j = 0; j < rank; ++j) {
        wh[j] = lam[j];
        wh[rank + j] = 1.0 - 1.0 / std::sqrt(lam[j] + 1.0);
    }
    // The new factors replace the old ones in place (the session orders this
    // stream after every earlier use of them).
    PCK(cudaMemcpyAsync(p->w, wh.data(), wh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(M, Sh.data(), Sh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    k_combine_rows<<<nblk((size_t)rank * N, 256), 256, 0, st>>>(M, Q, p->V, kk, rank, N);
    HV_RT_INTERNAL(launched("k_combine_rows"));
    k_combine_rows<<<nblk((size_t)rank * N, 256), 256, 0, st>>>(M, HQ, p->U, kk, rank, N);
    HV_RT_INTERNAL(launched("k_combine_rows"));
    PCK(cudaStreamSynchronize(st));
    p->r = rank;
    p->lam.assign(lam.begin(), lam.begin() + rank);
    return HV_OK;
}

extern "C" int hv_posterior_eigs(const hv_posterior *p, double *lambda, float *V, void *stream)
{
    if (!p) return hvi::fail(HV_EINVAL, "null posterior");
    if (lambda)
        for (int i = 0; i < p->r; ++i) lambda[i] = p->lam[i];
    if (V && p->r > 0)
        PCK(cudaMemcpyAsync(V, p->V, (size_t)p->r * p->nz * p->nx * sizeof(float), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return HV_OK;
}

extern "C" int hv_posterior_rank(const hv_posterior *p) { return p ? p->r : -1; }

extern "C" int hv_gpcn_propose(int n, int c, const float *m, const float *m_map, const float *zeta, double beta,
                               float *m_new, float *d_new, void *stream)
{
    if (n < 1 || c < 1 || c > 65535 || !m || !m_map || !zeta || !m_new)
        return hvi::fail(HV_EINVAL, "bad gpCN proposal arguments");
    if (!(beta > 0 && beta < 1)) return hvi::fail(HV_EINVAL, "beta = %g; need 0 < beta < 1", beta);
    k_gpcn_propose<<<dim3(nblk((size_t)n, 256), c), 256, 0, (cudaStream_t)stream>>>(
        m, m_map, zeta, (float)std::sqrt(1.0 - beta * beta), (float)beta, m_new, d_new, c, (size_t)n);
    return launched("k_gpcn_propose");
}

extern "C" int hv_gpcn_accept(int n, int c, const double *phi_new, const float *m_new, const float *d_new,
                              const float *Hd_new, const double *log_u, float *m, double *delta_cur, int *accepted,
                              void *stream)
{
    if (n < 1 || c < 1 || c > 65535 || !phi_new || !m_new || !d_new || !Hd_new || !log_u || !m || !delta_cur ||
        !accepted)
        return hvi::fail(HV_EINVAL, "bad gpCN acceptance arguments");
    cudaStream_t st = (cudaStream_t)stream;
    k_gpcn_decide<<<c, 256, 0, st>>>(phi_new, d_new, Hd_new, log_u, delta_cur, accepted, (size_t)n);
    HV_RT_INTERNAL(launched("k_gpcn_decide"));
    k_gpcn_take<<<dim3(nblk(n, 256), c), 256, 0, st>>>(m_new, accepted, m, (size_t)n);
    return launched("k_gpcn_take");
}
