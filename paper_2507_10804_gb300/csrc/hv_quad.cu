// hv_quad.cu -- the ideal quadratic test model (section 4.1).
//
// Misfit Hessian H_d = A A^T + V_r Lambda_r V_r^T (eq. (toy-hess)), A the
// order-1/2 PsiDO with the rank-3 symbol of eq. (toy-symbol)
//   s_A(x, xi) = w(x) P(|xi|) (0.1 + cos^2(arg xi + pi x / x_max)) / (0.1 + (z / z_max)^2)
//             = sum_k a_k(x) b_k(xi)           (compound-angle expansion),
// applied by the low-rank-symbol engine (hv_pdo.cu: A v = Re sum_k a_k F^-1 b_k F v,
// A^T by the transposed apply).  The objective is Phi_d(W m) plus the Matern
// prior: Phi(m) = 1/2 (W m - m*)^T H_d (W m - m*) + 1/2 m^T R m.
//
// Readings (the paper describes P, w and V_r only qualitatively):
//   P(rho) = (rho / rho_c)^(1/2) exp(-(rho / rho_c)^4), rho in rad/m;
//   w = W = product of 1D tapers sin^2(pi/2 (i + 1/2) / L) over L cells at each edge;
//   z = iz h, x = ix h, z_max = nz h, x_max = nx h, arg xi = atan2(xi_z, xi_x);
//   V_r: e^{-8 z / z_max} cos / sin(2 pi p x / x_max), p = 1 .. r/2, unit norm.
// The factor tables are evaluated once on the host in FP64 and stored in FP32.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

#define QCK(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

struct hv_quad {
    int device = -1;
    int nz = 0, nx = 0, nlr = 0, L = 0;
    double h = 0, rho_c = 0;
    hvk::LrSym lr;                 // a_k, b_k (r = 3) and the FFT engine
    float *W = nullptr;            // [N] window
    float *V = nullptr;            // [nlr][N] low-rank modes
    double *lam = nullptr;         // [nlr]
    hvk::Prior prior;
    float *t1 = nullptr, *t2 = nullptr;   // scratch, tk fields each
    double *c = nullptr;                  // scratch, tk * nlr coefficients
    double *red = nullptr;                // reduction partials, then 2 tk dot products
    int tk = 0;
    cudaEvent_t done = nullptr;
    std::mutex *mu = nullptr;
};

namespace {

unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

int launched(const char *what)
{
    hvk::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

// Elementwise kernels: grid (points / 256, k), no 64-bit division per element.
// out[q][e] = W[e] v[q][e]
__global__ void k_window(const float *__restrict__ W, const float *v, float *out, int k, size_t N)   // out may be v
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const size_t t = (size_t)blockIdx.y * N + e;
    out[t] = W[e] * v[t];
}

// e[q] = W m[q] - m*[q]  (mstar broadcast when it holds one field)
__global__ void k_residual_field(const float *__restrict__ W, const float *__restrict__ m,
                                 const float *__restrict__ mstar, float *__restrict__ e, int k, size_t N,
                                 bool one_target)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const size_t t = (size_t)blockIdx.y * N + i;
    e[t] = fmaf(W[i], m[t], -mstar[one_target ? i : t]);
}

__global__ void k_add2(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out, int k)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = a[i] + b[i];
}

// grad[q] = W He[q] + Rm[q]
__global__ void k_grad(const float *__restrict__ W, const float *__restrict__ He, const float *__restrict__ Rm,
                       float *__restrict__ g, int k, size_t N)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const size_t t = (size_t)blockIdx.y * N + i;
    g[t] = fmaf(W[i], He[t], Rm[t]);
}

std::vector<double> taper(int n, int L)
{
    std::vector<double> left(n, 1.0), t(n);
    for (int i = 0; i < n && i < L; ++i) {
        const double s = std::sin(0.5 * M_PI * (i + 0.5) / L);
        left[i] = s * s;
    }
    for (int i = 0; i < n; ++i) t[i] = std::min(left[i], left[n - 1 - i]);
    return t;
}

int signed_index(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

int grow(hv_quad *q, int k)
{
    if (q->tk >= k) return HV_OK;
    cudaFree(q->t1);   // synchronises: earlier work on the old scratch is done
    cudaFree(q->t2);
    cudaFree(q->c);
    cudaFree(q->red);
    q->t1 = q->t2 = nullptr;
    q->c = q->red = nullptr;
    q->tk = 0;
    const size_t N = (size_t)q->nz * q->nx;
    const size_t nred = std::max(hvk::coef_scratch(std::max(q->nlr, 1), k, N), hvk::rows_dot_scratch(k, N)) + 2 * (size_t)k;
    cudaError_t e;
    if ((e = cudaMalloc(&q->t1, (size_t)k * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&q->t2, (size_t)k * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&q->c, (size_t)k * std::max(q->nlr, 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&q->red, nred * sizeof(double))) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "quadratic-model scratch: %s", cudaGetErrorString(e));
    q->tk = k;
    return HV_OK;
}

// out = (A A^T + V Lambda V^T) v for k fields (out may not alias v); uses t2.
int hd_raw(hv_quad *q, const float *v, int k, float *out, cudaStream_t st)
{
    const size_t N = (size_t)q->nz * q->nx;
    HV_RT_INTERNAL(hvk::lr_apply(q->lr, v, k, q->t2, st, hvk::kLrTranspose));
    HV_RT_INTERNAL(hvk::lr_apply(q->lr, q->t2, k, out, st, hvk::kLrForward));
    if (q->nlr > 0) {   // + V Lambda V^T v
        HV_RT_INTERNAL(hvk::coef(q->V, q->nlr, v, k, N, q->lam, q->c, q->red, st));
        HV_RT_INTERNAL(hvk::combine(q->V, q->nlr, q->c, k, N, out, 1.0f, out, st));
    }
    return HV_OK;
}

int quad_op(void *ctx, const float *v, int k, float *out, void *stream)
{
    return hv_quad_apply(static_cast<hv_quad *>(ctx), HV_QUAD_HD, v, k, out, stream);
}

}  // namespace

extern "C" int hv_quad_create(int nz, int nx, double h, double rho_c, int taper_cells, int nlr, const double *lam,
                              double delta, double gamma, hv_quad **out)
{
    if (out) *out = nullptr;
    if (!out) return hvi::fail(HV_EINVAL, "null output");
    if (nz < 4 || nx < 4 || !(h > 0)) return hvi::fail(HV_EINVAL, "grid %d x %d, h = %g; need nz, nx >= 4, h > 0", nz, nx, h);
    if (!(rho_c > 0)) return hvi::fail(HV_EINVAL, "rho_c must be > 0");
    if (taper_cells < 0 || 2 * taper_cells > std::min(nz, nx)) return hvi::fail(HV_EINVAL, "taper of %d cells", taper_cells);
    if (nlr < 0 || nlr % 2 || nlr / 2 >= nx / 2 || (nlr > 0 && !lam))
        return hvi::fail(HV_EINVAL, "nlr = %d; need an even count with nlr / 2 < nx / 2 and its eigenvalues", nlr);
    for (int j = 0; j < nlr; ++j)
        if (!(lam[j] >= 0)) return hvi::fail(HV_EINVAL, "eigenvalue %d of the low-rank part is negative", j);
    int dev = -1;
    QCK(cudaGetDevice(&dev));
    hv_quad *q = new hv_quad;
    q->device = dev;
    q->nz = nz;
    q->nx = nx;
    q->nlr = nlr;
    q->L = taper_cells;
    q->h = h;
    q->rho_c = rho_c;
    q->mu = new std::mutex;
    const size_t N = (size_t)nz * nx;
    auto fail = [&](int rc) {
        hv_quad_destroy(q);
        return rc;
    };
    // tables in FP64 on the host
    const std::vector<double> tz = taper(nz, taper_cells), tx = taper(nx, taper_cells);
    std::vector<float> W(N), V((size_t)nlr * N);
    std::vector<float2> a(3 * N), b(3 * N);
    for (int i = 0; i < nz; ++i) {
        const double zr = (double)i / nz, den = 1.0 / (0.1 + zr * zr);
        for (int j = 0; j < nx; ++j) {
            const double w = tz[i] * tx[j], xr = (double)j / nx;
            const size_t e = (size_t)i * nx + j;
            W[e] = (float)w;
            a[e] = make_float2((float)(w * den), 0.0f);
            a[N + e] = make_float2((float)(w * den * std::cos(2.0 * M_PI * xr)), 0.0f);
            a[2 * N + e] = make_float2((float)(w * den * std::sin(2.0 * M_PI * xr)), 0.0f);
            const double fz = 2.0 * M_PI * signed_index(i, nz) / (nz * h);
            const double fx = 2.0 * M_PI * signed_index(j, nx) / (nx * h);
            const double r = std::hypot(fz, fx) / rho_c, P = std::sqrt(r) * std::exp(-r * r * r * r);
            const double ang = std::atan2(fz, fx);
            b[e] = make_float2((float)(0.6 * P), 0.0f);
            b[N + e] = make_float2((float)(0.5 * std::cos(2.0 * ang) * P), 0.0f);
            b[2 * N + e] = make_float2((float)(-0.5 * std::sin(2.0 * ang) * P), 0.0f);
        }
    }
    std::vector<double> dz(nz);
    double nd = 0.0;
    for (int i = 0; i < nz; ++i) {
        dz[i] = std::exp(-8.0 * i / nz);
        nd += dz[i] * dz[i];
    }
    for (int p = 1; p <= nlr / 2; ++p)
        for (int f = 0; f < 2; ++f) {
            std::vector<double> cx(nx);
            double nc = 0.0;
            for (int j = 0; j < nx; ++j) {
                const double ph = 2.0 * M_PI * p * j / nx;
                cx[j] = f == 0 ? std::cos(ph) : std::sin(ph);
                nc += cx[j] * cx[j];
            }
            const double s = 1.0 / std::sqrt(nd * nc);
            float *vj = V.data() + (size_t)(2 * (p - 1) + f) * N;
            for (int i = 0; i < nz; ++i)
                for (int j = 0; j < nx; ++j) vj[(size_t)i * nx + j] = (float)(s * dz[i] * cx[j]);
        }
    hvk::LrGeo g;
    g.nz = nz;
    g.nx = nx;
    g.r = 3;
    g.h = h;
    int rc = hvk::lr_create(q->lr, g);
    if (rc != HV_OK) return fail(rc);
    rc = hvk::prior_create(q->prior, nz, nx, h, delta, gamma);
    if (rc != HV_OK) return fail(rc);
    cudaError_t e;
    if ((e = cudaMalloc(&q->W, N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&q->V, std::max<size_t>(V.size(), 1) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&q->lam, std::max(nlr, 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMemcpy(q->W, W.data(), N * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(q->lr.a, a.data(), a.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(q->lr.b, b.data(), b.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (nlr > 0 && (e = cudaMemcpy(q->V, V.data(), V.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (nlr > 0 && (e = cudaMemcpy(q->lam, lam, nlr * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess))
        return fail(hvi::fail(HV_ECUDA, "quadratic model tables: %s", cudaGetErrorString(e)));
    *out = q;
    return HV_OK;
}

extern "C" int hv_quad_destroy(hv_quad *q)
{
    if (!q) return HV_OK;
    if (q->done) cudaEventSynchronize(q->done);
    if (q->lr.done) cudaEventSynchronize(q->lr.done);
    hvk::lr_destroy(q->lr);
    hvk::prior_destroy(q->prior);
    cudaFree(q->W);
    cudaFree(q->V);
    cudaFree(q->lam);
    cudaFree(q->t1);
    cudaFree(q->t2);
    cudaFree(q->c);
    cudaFree(q->red);
    if (q->done) cudaEventDestroy(q->done);
    delete q->mu;
    delete q;
    return HV_OK;
}

extern "C" int hv_quad_apply(hv_quad *q, int op, const float *v, int k, float *out, void *stream)
{
    if (!q || !v || !out) return hvi::fail(HV_EINVAL, "null model, vector or output");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "k = %d vectors; need 1 <= k <= 65535", k);
    if (op < HV_QUAD_HD || op > HV_QUAD_HD_RAW) return hvi::fail(HV_EINVAL, "unknown quadratic-model operator %d", op);
    int dev = -1;
    QCK(cudaGetDevice(&dev));
    if (dev != q->device) return hvi::fail(HV_EINVAL, "current device %d is not the model's device %d", dev, q->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)q->nz * q->nx;
    std::lock_guard<std::mutex> lk(*q->mu);
    QCK(cudaStreamWaitEvent(st, q->done, 0));
    HV_RT_INTERNAL(grow(q, k));
    if (op == HV_QUAD_A) {
        HV_RT_INTERNAL(hvk::lr_apply(q->lr, v, k, out, st, hvk::kLrForward));
    } else if (op == HV_QUAD_AT) {
        HV_RT_INTERNAL(hvk::lr_apply(q->lr, v, k, out, st, hvk::kLrTranspose));
    } else if (op == HV_QUAD_HD_RAW) {
        HV_RT_INTERNAL(hd_raw(q, v, k, out, st));
    } else {   // W (A A^T + V Lambda V^T) W v
        k_window<<<dim3(nblk(N, 256), k), 256, 0, st>>>(q->W, v, q->t1, k, N);
        HV_RT_INTERNAL(launched("k_window"));
        HV_RT_INTERNAL(hd_raw(q, q->t1, k, out, st));
        k_window<<<dim3(nblk(N, 256), k), 256, 0, st>>>(q->W, out, out, k, N);
        HV_RT_INTERNAL(launched("k_window"));
    }
    QCK(cudaEventRecord(q->done, st));
    return HV_OK;
}

extern "C" int hv_quad_objective(hv_quad *q, const float *m, const float *mstar, int k, int one_target, double *phi,
                                 float *grad, void *stream)
{
    if (!q || !m || !mstar || !phi) return hvi::fail(HV_EINVAL, "null model, states, target or output");
    if (k < 1 || k > 65535) return hvi::fail(HV_EINVAL, "k = %d states; need 1 <= k <= 65535", k);
    int dev = -1;
    QCK(cudaGetDevice(&dev));
    if (dev != q->device) return hvi::fail(HV_EINVAL, "current device %d is not the model's device %d", dev, q->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)q->nz * q->nx;
    std::lock_guard<std::mutex> lk(*q->mu);
    QCK(cudaStreamWaitEvent(st, q->done, 0));
    // t1: the residual e, then R m; He in a scratch of its own
    HV_RT_INTERNAL(grow(q, 2 * k));
    float *e = q->t1, *Rm = q->t1 + (size_t)k * N, *He = q->t2 + (size_t)k * N;
    k_residual_field<<<dim3(nblk(N, 256), k), 256, 0, st>>>(q->W, m, mstar, e, k, N, one_target != 0);
    HV_RT_INTERNAL(launched("k_residual_field"));
    HV_RT_INTERNAL(hd_raw(q, e, k, He, st));
    HV_RT_INTERNAL(hvk::prior_R(q->prior, m, Rm, k, st));
    // phi = 1/2 e.He + 1/2 m.Rm (FP64)
    double *s1 = q->red + hvk::rows_dot_scratch(k, N) + 0, *s2 = s1 + k;
    HV_RT_INTERNAL(hvk::rows_dot(e, He, s1, k, N, 0.5, q->red, st));
    HV_RT_INTERNAL(hvk::rows_dot(m, Rm, s2, k, N, 0.5, q->red, st));
    k_add2<<<nblk(k, 128), 128, 0, st>>>(s1, s2, phi, k);
    HV_RT_INTERNAL(launched("k_add2"));
    if (grad) {
        k_grad<<<dim3(nblk(N, 256), k), 256, 0, st>>>(q->W, He, Rm, grad, k, N);
        HV_RT_INTERNAL(launched("k_grad"));
    }
    QCK(cudaEventRecord(q->done, st));
    return HV_OK;
}

extern "C" int hv_quad_tables(const hv_quad *q, float *a, float *b, float *V, float *W, void *stream)
{
    if (!q) return hvi::fail(HV_EINVAL, "null model");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)q->nz * q->nx;
    if (a) QCK(cudaMemcpyAsync(a, q->lr.a, 3 * N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (b) QCK(cudaMemcpyAsync(b, q->lr.b, 3 * N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (V && q->nlr > 0) QCK(cudaMemcpyAsync(V, q->V, q->nlr * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (W) QCK(cudaMemcpyAsync(W, q->W, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HV_OK;
}

extern "C" int hv_quad_operator(hv_quad *q, hv_operator *op)
{
    if (!q || !op) return hvi::fail(HV_EINVAL, "null model or operator");
    op->nz = q->nz;
    op->nx = q->nx;
    op->h = q->h;
    op->apply = quad_op;
    op->ctx = q;
    return HV_OK;
}
