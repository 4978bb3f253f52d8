// hv_highpass.cu -- the high-pass filter applied to the Hessian before the
// PSF and PDO approximations (sections 3.2 and 3.7: the low-frequency part of
// H_d spoils the locality of the point spread functions and the spectral
// separation of the probing, so it is removed before approximating).
//
// F_hp v = Re F^-1 (phi(|xi|) F v) on the periodic DFT of the nz x nx grid,
// phi(rho) = 1 - exp(-rho^2 / (2 rho_c^2)), xi = (2 pi k_z / (nz h),
// 2 pi k_x / (nx h)) for the signed indices; the approximations are built from
// F_hp H_d F_hp (both sides, so the operator stays symmetric).  The transforms
// are real-to-complex and back (cuFFT, FP32); the multiplier is tabulated in
// FP64 on the host and stored in FP32 with the 1 / (nz nx) scale folded in.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace hvk {

namespace {

// spec[q][e] *= tab[e], e over the nz x (nx/2 + 1) half spectrum, q < k.
__global__ void k_hp_scale(float2 *__restrict__ spec, const float *__restrict__ tab, size_t n, int k)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float t = tab[e];
    for (int q = 0; q < k; ++q) {
        float2 v = spec[(size_t)q * n + e];
        v.x *= t;
        v.y *= t;
        spec[(size_t)q * n + e] = v;
    }
}

int fft_ok(cufftResult r, const char *what)
{
    if (r != CUFFT_SUCCESS) return hvi::fail(HV_ECUDA, "%s failed (cuFFT %d)", what, (int)r);
    return HV_OK;
}

}  // namespace

int highpass_create(Highpass &F, int nz, int nx, double h, double rho_c, int kmax)
{
    if (nz < 2 || nx < 2 || !(h > 0) || !(rho_c > 0) || kmax < 1)
        return hvi::fail(HV_EINVAL, "high-pass filter: grid %d x %d, h %g, rho_c %g, k %d", nz, nx, h, rho_c, kmax);
    F.nz = nz;
    F.nx = nx;
    F.kmax = kmax;
    F.h = h;
    F.rho_c = rho_c;
    const int nh = nx / 2 + 1;
    const size_t n = (size_t)nz * nh;
    std::vector<float> tab(n);
    const double pi = 3.14159265358979323846;
    for (int iz = 0; iz < nz; ++iz) {
        const int kz = iz <= nz / 2 ? iz : iz - nz;
        const double xz = 2.0 * pi * kz / (nz * h);
        for (int ix = 0; ix < nh; ++ix) {
            const double xx = 2.0 * pi * ix / (nx * h);
            const double r2 = xz * xz + xx * xx;
            tab[(size_t)iz * nh + ix] = (float)((1.0 - std::exp(-r2 / (2.0 * rho_c * rho_c))) / ((double)nz * nx));
        }
    }
    cudaError_t e;
    if ((e = cudaMalloc(&F.tab, n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&F.spec, (size_t)kmax * n * sizeof(float2))) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "high-pass filter: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpy(F.tab, tab.data(), n * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return hvi::fail(HV_ECUDA, "high-pass filter: %s", cudaGetErrorString(e));
    int dims[2] = {nz, nx};
    HV_RT_INTERNAL(fft_ok(cufftPlanMany(&F.fwd, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, kmax), "cufftPlanMany"));
    F.fwd_ok = true;
    HV_RT_INTERNAL(fft_ok(cufftPlanMany(&F.inv, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, kmax), "cufftPlanMany"));
    F.inv_ok = true;
    HV_RT_INTERNAL(fft_ok(cufftPlan2d(&F.fwd1, nz, nx, CUFFT_R2C), "cufftPlan2d"));
    F.fwd1_ok = true;
    HV_RT_INTERNAL(fft_ok(cufftPlan2d(&F.inv1, nz, nx, CUFFT_C2R), "cufftPlan2d"));
    F.inv1_ok = true;
    return HV_OK;
}

void highpass_destroy(Highpass &F)
{
    if (F.fwd_ok) cufftDestroy(F.fwd);
    if (F.inv_ok) cufftDestroy(F.inv);
    if (F.fwd1_ok) cufftDestroy(F.fwd1);
    if (F.inv1_ok) cufftDestroy(F.inv1);
    cudaFree(F.tab);
    cudaFree(F.spec);
    F = Highpass{};
}

// out = F_hp v for k fields (out may be v): whole batches of kmax fields with
// the batched plans, the rest one field at a time (a plan reads and writes
// exactly its batch).
int highpass_apply(Highpass &F, const float *v, int k, float *out, cudaStream_t st)
{
    const size_t N = (size_t)F.nz * F.nx, n = (size_t)F.nz * (F.nx / 2 + 1);
    for (cufftHandle p : {F.fwd, F.inv, F.fwd1, F.inv1}) HV_RT_INTERNAL(fft_ok(cufftSetStream(p, st), "cufftSetStream"));
    for (int q0 = 0; q0 < k;) {
        const bool whole = k - q0 >= F.kmax;
        const int kb = whole ? F.kmax : 1;
        HV_RT_INTERNAL(fft_ok(cufftExecR2C(whole ? F.fwd : F.fwd1, const_cast<float *>(v + (size_t)q0 * N), F.spec),
                              "cufftExecR2C"));
        k_hp_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F.spec, F.tab, n, kb);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "k_hp_scale: %s", cudaGetErrorString(e));
        HV_RT_INTERNAL(fft_ok(cufftExecC2R(whole ? F.inv : F.inv1, F.spec, out + (size_t)q0 * N), "cufftExecC2R"));
        q0 += kb;
    }
    return HV_OK;
}

}  // namespace hvk
