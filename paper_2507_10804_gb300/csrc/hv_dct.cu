// hv_dct.cu -- the inverse of the Matern prior's operator A = delta I - gamma Lap_h
// (section 2.1) by a fast transform: A is diagonal in the 2D DCT-II basis
// (homogeneous Neumann conditions, mirror ghost cells), A^-1 v = C^T diag(1 /
// lambda) C v with lambda_kl = delta + gamma (4 / h^2)(sin^2(pi k / (2 nz)) +
// sin^2(pi l / (2 nx))).
//
// The unnormalised 2D DCT-II X of v comes from one real 2D DFT of the
// reordered field w[j1][j2] = v[p(j1)][q(j2)], p(j) = 2j for the first
// ceil(n/2) indices and 2(n - 1 - j) + 1 for the rest (the reordering of
// Makhoul, 1980): with Z(a, b) = e^{-i pi a / (2 nz)} e^{-i pi b / (2 nx)} W(a, b),
//   X(a, b) = 1/2 (Re Z(a, b) - Im Z(a, nx - b)),
// and back, W(a, b) = e^{i pi a / (2 nz)} e^{i pi b / (2 nx)} (X(a, b) - X(nz - a, nx - b)
//   - i (X(nz - a, b) + X(a, nx - b))), X = 0 at index nz or nx.
// The orthonormal scale factors cancel between the forward and the inverse
// transform, so A^-1 v is the inverse of (X / lambda): one real-to-complex
// transform, one kernel that forms X, divides by lambda and rebuilds the half
// spectrum, and one complex-to-real transform (cuFFT, FP32).
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

namespace hvk {

namespace {

__device__ __forceinline__ int perm_index(int j, int n)
{
    const int h = (n + 1) / 2;
    return j < h ? 2 * j : 2 * (n - 1 - j) + 1;
}

// forward: w[q][j1][j2] = v[q][p(j1)][q(j2)]; inverse: out[q][p(j1)][q(j2)] = w[q][j1][j2].
__global__ void k_dct_perm(const float *__restrict__ in, float *__restrict__ out, int n1, int n2, int inverse)
{
    const int j2 = blockIdx.x * blockDim.x + threadIdx.x, j1 = blockIdx.y;
    if (j2 >= n2) return;
    const size_t base = (size_t)blockIdx.z * n1 * n2;
    const size_t a = base + (size_t)j1 * n2 + j2, b = base + (size_t)perm_index(j1, n1) * n2 + perm_index(j2, n2);
    if (inverse) out[b] = in[a];
    else out[a] = in[b];
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// The half spectrum of A^-1 v from that of v (the two buffers differ): one
// thread per (a, c), c <= n2 / 2; grid (ceil((n2/2 + 1) / 128), n1, k).
// tw1[a] = (cos, sin)(pi a / (2 n1)) for a <= n1, tw2 likewise for n2; inv[a][b]
// = 1 / (lambda_ab n1 n2).
__global__ void k_dct_scale(const float2 *__restrict__ Wh, float2 *__restrict__ Wo, const float2 *__restrict__ tw1,
                            const float2 *__restrict__ tw2, const float *__restrict__ inv, int n1, int n2)
{
    const int h2 = n2 / 2 + 1;
    const int c = blockIdx.x * blockDim.x + threadIdx.x, a = blockIdx.y;
    if (c >= h2) return;
    const size_t base = (size_t)blockIdx.z * n1 * h2;
    auto W = [&](int x, int y) {            // the full spectrum from its half: W(-x, -y) = conj W(x, y)
        x = ((x % n1) + n1) % n1;
        y = ((y % n2) + n2) % n2;
        if (y < h2) return Wh[base + (size_t)x * h2 + y];
        return conj2(Wh[base + (size_t)((n1 - x) % n1) * h2 + (n2 - y)]);
    };
    auto Z = [&](int x, int y) { return cmul(conj2(tw1[x]), cmul(conj2(tw2[y]), W(x, y))); };
    auto X = [&](int x, int y) {            // x <= n1, y <= n2; zero at the index n
        if (x >= n1 || y >= n2) return 0.0f;
        const float2 z1 = Z(x, y), z2 = Z(x, n2 - y);
        return 0.5f * (z1.x - z2.y) * inv[(size_t)x * n2 + y];
    };
    const float A = X(a, c), B = a > 0 ? X(n1 - a, c) : 0.0f, C = c > 0 ? X(a, n2 - c) : 0.0f,
                D = (a > 0 && c > 0) ? X(n1 - a, n2 - c) : 0.0f;
    Wo[base + (size_t)a * h2 + c] = cmul(tw1[a], cmul(tw2[c], make_float2(A - D, -(B + C))));
}

// out = v * s[0] (the 1 x 1 grid).
__global__ void k_scale_by(const float *__restrict__ v, const float *__restrict__ s, float *__restrict__ out)
{
    out[0] = v[0] * s[0];
}

int fft_check(cufftResult r, const char *what)
{
    if (r != CUFFT_SUCCESS) return hvi::fail(HV_ECUDA, "%s failed (cuFFT %d)", what, (int)r);
    return HV_OK;
}

int plan(cufftHandle *p, int n1, int n2, cufftType t, int batch)
{
    if (n1 == 1) {
        int n = n2;
        return fft_check(cufftPlanMany(p, 1, &n, nullptr, 1, 0, nullptr, 1, 0, t, batch), "cufftPlanMany");
    }
    int dims[2] = {n1, n2};
    return fft_check(cufftPlanMany(p, 2, dims, nullptr, 1, 0, nullptr, 1, 0, t, batch), "cufftPlanMany");
}

}  // namespace

int dct_create(Dct2 &D, int nz, int nx, double h, double delta, double gamma, int kmax)
{
    if (nz < 1 || nx < 1 || kmax < 1) return hvi::fail(HV_EINVAL, "DCT: grid %d x %d, k %d", nz, nx, kmax);
    // A field with one column is stored like a field with one row: transform it as 1 x nz.
    const bool swap = nx == 1 && nz > 1;
    D.n1 = swap ? 1 : nz;
    D.n2 = swap ? nz : nx;
    D.kmax = kmax;
    const int n1 = D.n1, n2 = D.n2, h2 = n2 / 2 + 1;
    const double pi = 3.14159265358979323846;
    std::vector<float2> tw((size_t)n1 + 1 + n2 + 1);
    for (int a = 0; a <= n1; ++a) tw[a] = make_float2((float)std::cos(pi * a / (2.0 * n1)), (float)std::sin(pi * a / (2.0 * n1)));
    for (int b = 0; b <= n2; ++b)
        tw[n1 + 1 + b] = make_float2((float)std::cos(pi * b / (2.0 * n2)), (float)std::sin(pi * b / (2.0 * n2)));
    std::vector<float> inv((size_t)nz * nx);
    for (int k = 0; k < nz; ++k)
        for (int l = 0; l < nx; ++l) {
            const double sz = std::sin(pi * k / (2.0 * nz)), sx = std::sin(pi * l / (2.0 * nx));
            const double lam = delta + gamma * (4.0 / (h * h)) * (sz * sz + sx * sx);
            inv[(size_t)k * nx + l] = (float)(1.0 / (lam * (double)nz * nx));   // [nz][nx] = [n1][n2] in memory
        }
    cudaError_t e;
    const size_t N = (size_t)nz * nx, S = (size_t)n1 * h2;
    if ((e = cudaMalloc(&D.tw, tw.size() * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&D.inv, N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&D.w, (size_t)kmax * N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&D.s1, (size_t)kmax * S * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&D.s2, (size_t)kmax * S * sizeof(float2))) != cudaSuccess ||
        (e = cudaMemcpy(D.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(D.inv, inv.data(), N * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "DCT tables: %s", cudaGetErrorString(e));
    if (N == 1) return HV_OK;                  // one point: A^-1 is a scale, no transform
    HV_RT_INTERNAL(plan(&D.f, n1, n2, CUFFT_R2C, kmax));
    D.f_ok = true;
    HV_RT_INTERNAL(plan(&D.i, n1, n2, CUFFT_C2R, kmax));
    D.i_ok = true;
    HV_RT_INTERNAL(plan(&D.f1, n1, n2, CUFFT_R2C, 1));
    D.f1_ok = true;
    HV_RT_INTERNAL(plan(&D.i1, n1, n2, CUFFT_C2R, 1));
    D.i1_ok = true;
    return HV_OK;
}

void dct_destroy(Dct2 &D)
{
    if (D.f_ok) cufftDestroy(D.f);
    if (D.i_ok) cufftDestroy(D.i);
    if (D.f1_ok) cufftDestroy(D.f1);
    if (D.i1_ok) cufftDestroy(D.i1);
    cudaFree(D.tw);
    cudaFree(D.inv);
    cudaFree(D.w);
    cudaFree(D.s1);
    cudaFree(D.s2);
    D = Dct2{};
}

// out = A^-1 v for k fields (out may be v): whole batches of kmax fields with
// the batched plans, the rest one field at a time.
int dct_apply(Dct2 &D, const float *v, int k, float *out, cudaStream_t st)
{
    const int n1 = D.n1, n2 = D.n2, h2 = n2 / 2 + 1;
    const size_t N = (size_t)n1 * n2;
    if (N == 1) {                               // a 1 x 1 grid: the transform is the identity
        for (int q = 0; q < k; ++q) {
            k_scale_by<<<1, 1, 0, st>>>(v + q, D.inv, out + q);
            count_launch();
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? HV_OK : hvi::fail(HV_ECUDA, "k_scale_by: %s", cudaGetErrorString(e));
    }
    for (cufftHandle p : {D.f, D.i, D.f1, D.i1}) HV_RT_INTERNAL(fft_check(cufftSetStream(p, st), "cufftSetStream"));
    for (int q0 = 0; q0 < k;) {
        const bool whole = k - q0 >= D.kmax;
        const int kb = whole ? D.kmax : 1;
        const dim3 gp((unsigned)((n2 + 127) / 128), (unsigned)n1, (unsigned)kb);
        k_dct_perm<<<gp, 128, 0, st>>>(v + (size_t)q0 * N, D.w, n1, n2, 0);
        count_launch();
        HV_RT_INTERNAL(fft_check(cufftExecR2C(whole ? D.f : D.f1, D.w, D.s1), "cufftExecR2C"));
        k_dct_scale<<<dim3((unsigned)((h2 + 127) / 128), (unsigned)n1, (unsigned)kb), 128, 0, st>>>(
            D.s1, D.s2, D.tw, D.tw + n1 + 1, D.inv, n1, n2);
        count_launch();
        HV_RT_INTERNAL(fft_check(cufftExecC2R(whole ? D.i : D.i1, D.s2, D.w), "cufftExecC2R"));
        k_dct_perm<<<gp, 128, 0, st>>>(D.w, out + (size_t)q0 * N, n1, n2, 1);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "DCT kernels: %s", cudaGetErrorString(e));
        q0 += kb;
    }
    return HV_OK;
}

}  // namespace hvk
