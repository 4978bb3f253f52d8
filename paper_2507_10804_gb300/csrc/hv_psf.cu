// hv_psf.cu -- point-spread-function approximation of the misfit Hessian:
// impulse batches, PSF extraction and the approximate apply (section 3.2, and
// the PsiDO row form of section 3.5).
//
// Sample points form a lattice of spacing S cells on the interior grid (first
// point at (S/2, S/2)), split into B x B interleaved batches.  One batched
// Hessian application to the batches' impulse sums gives every PSF:
//   p_k(d) = (H v_batch(k))[x_k + d],  |d|_inf <= R = (B S - 1) / 2
// (zero where x_k + d leaves the grid).  The approximation interpolates these
// symbol rows with bilinear weights on the lattice,
//   (H~ v)(x) = sum_k w_k(x) sum_d p_k(d) v(x + d),
// which is (2 pi)^2 sum_k D_{w_k} F^-1 D_{conj(p_k^)} F v evaluated in space:
// the rows are compactly supported, so the correlation costs 4 (2R+1)^2
// multiply-adds per point instead of one inverse FFT per sample point.
#include "hv_internal.h"

namespace hvk {

namespace {

__global__ void k_psf_impulses(float *v, PsfGeo g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.na * g.nb) return;
    const int a = k / g.nb, b = k - a * g.nb;
    const int q = (a % g.B) * g.B + (b % g.B);
    v[((size_t)q * g.nz + g.cz0 + g.S * a) * g.nx + g.cx0 + g.S * b] = 1.0f;
}

__global__ void k_psf_extract(const float *__restrict__ Hv, float *__restrict__ psf, PsfGeo g)
{
    const int W = 2 * g.R + 1;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)g.na * g.nb * W * W) return;
    const int k = (int)(i / ((size_t)W * W));
    const int rem = (int)(i - (size_t)k * W * W);
    const int dz = rem / W - g.R, dx = rem % W - g.R;
    const int a = k / g.nb, b = k - a * g.nb;
    const int q = (a % g.B) * g.B + (b % g.B);
    const int z = g.cz0 + g.S * a + dz, x = g.cx0 + g.S * b + dx;
    psf[i] = (z >= 0 && z < g.nz && x >= 0 && x < g.nx) ? Hv[((size_t)q * g.nz + z) * g.nx + x] : 0.0f;
}

// Lattice interval [a0, a1] around grid index i along one axis and the weight
// f of a1 (a0 gets 1 - f); beyond the outermost points the index is clamped.
__device__ __forceinline__ void axis_weights(int i, int c0, int S, int n, int &a0, int &a1, float &f)
{
    int q = i - c0;
    q = max(q, 0);
    q = min(q, (n - 1) * S);
    a0 = min(q / S, max(n - 2, 0));
    a1 = min(a0 + 1, n - 1);
    f = (float)(q - a0 * S) / (float)S;
}

constexpr int kApplyT = 16;   // 16 x 16 outputs per CTA, one per thread

// out_j(x) = sum over the (up to 4) lattice points around x of w_k(x) times the
// correlation of v_j with p_k at x.  grid = (x tiles, z tiles, vectors).
__global__ void __launch_bounds__(kApplyT *kApplyT) k_psf_apply(const float *__restrict__ psf,
                                                                 const float *__restrict__ v,
                                                                 float *__restrict__ out, PsfGeo g)
{
    extern __shared__ float sv[];   // (T + 2R)^2 patch of v_j around the tile (zero off the grid)
    const int R = g.R, W = 2 * R + 1, PW = kApplyT + 2 * R;
    const int z0 = blockIdx.y * kApplyT, x0 = blockIdx.x * kApplyT, j = blockIdx.z;
    const float *vj = v + (size_t)j * g.nz * g.nx;
    for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
        const int z = z0 - R + i / PW, x = x0 - R + i % PW;
        sv[i] = (z >= 0 && z < g.nz && x >= 0 && x < g.nx) ? vj[(size_t)z * g.nx + x] : 0.0f;
    }
    __syncthreads();
    const int tz = threadIdx.x / kApplyT, tx = threadIdx.x % kApplyT;
    const int iz = z0 + tz, ix = x0 + tx;
    if (iz >= g.nz || ix >= g.nx) return;
    int a[2], b[2];
    float fz, fx;
    axis_weights(iz, g.cz0, g.S, g.na, a[0], a[1], fz);
    axis_weights(ix, g.cx0, g.S, g.nb, b[0], b[1], fx);
    const float wa[2] = {1.0f - fz, fz}, wb[2] = {1.0f - fx, fx};
    float acc = 0.0f;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            const float w = wa[p] * wb[q];
            if (w == 0.0f) continue;
            const float *pk = psf + (size_t)(a[p] * g.nb + b[q]) * W * W;
            float c = 0.0f;
            for (int dz = 0; dz < W; ++dz) {
                const float *row = sv + (tz + dz) * PW + tx;
                const float *prow = pk + dz * W;
                float r = 0.0f;
                for (int dx = 0; dx < W; ++dx) r = fmaf(__ldg(prow + dx), row[dx], r);
                c += r;
            }
            acc = fmaf(w, c, acc);
        }
    out[(size_t)j * g.nz * g.nx + (size_t)iz * g.nx + ix] = acc;
}

int check_launch(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

}  // namespace

int psf_apply_smem_bytes(int R) { return (kApplyT + 2 * R) * (kApplyT + 2 * R) * (int)sizeof(float); }

int launch_psf_impulses(const PsfGeo &g, float *v, cudaStream_t st)
{
    const int r = g.na * g.nb;
    k_psf_impulses<<<(r + 127) / 128, 128, 0, st>>>(v, g);
    return check_launch("k_psf_impulses");
}

int launch_psf_extract(const PsfGeo &g, const float *Hv, float *psf, cudaStream_t st)
{
    const size_t n = (size_t)g.na * g.nb * (2 * g.R + 1) * (2 * g.R + 1);
    k_psf_extract<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hv, psf, g);
    return check_launch("k_psf_extract");
}

int launch_psf_apply(const PsfGeo &g, const float *psf, const float *v, int k, float *out, cudaStream_t st)
{
    const int smem = psf_apply_smem_bytes(g.R);
    if (smem > 48 * 1024) return hvi::fail(HV_EINVAL, "window radius %d too large for the apply kernel", g.R);
    dim3 grid((g.nx + kApplyT - 1) / kApplyT, (g.nz + kApplyT - 1) / kApplyT, k);
    k_psf_apply<<<grid, kApplyT * kApplyT, smem, st>>>(psf, v, out, g);
    return check_launch("k_psf_apply");
}

}  // namespace hvk
