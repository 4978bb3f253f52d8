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

#include <algorithm>
#include <mutex>

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

// Lattice cells along one axis.  Cell 0 holds the indices before the first
// sample point (weight 1 on point 0), cell c = 1..n-1 the indices from point
// c-1 up to point c (weights 1 - f and f, f = (i - point c-1) / S), cell n the
// indices from the last point on (weight 1 on point n-1): the bilinear hat
// weights with constant extrapolation, cut where the set of points changes.
struct CellAxis {
    int lo, hi;      // indices [lo, hi)
    int p0, np;      // first lattice point and how many (1 or 2)
    int base;        // grid index of point p0
};

__device__ __forceinline__ CellAxis cell_axis(int c, int c0, int S, int n, int N)
{
    CellAxis a;
    if (c == 0) {
        a.lo = 0; a.hi = min(c0, N); a.p0 = 0; a.np = 1;
    } else if (c < n) {
        a.lo = c0 + (c - 1) * S; a.hi = c0 + c * S; a.p0 = c - 1; a.np = 2;
    } else {
        a.lo = c0 + (n - 1) * S; a.hi = N; a.p0 = n - 1; a.np = 1;
    }
    a.base = c0 + a.p0 * S;
    return a;
}

// Weights of the cell's points at index i: w[0] for p0, w[1] for p0 + 1.
__device__ __forceinline__ void cell_weights(const CellAxis &a, int i, int S, float (&w)[2])
{
    if (a.np == 2) {
        const float f = (float)(i - a.base) / (float)S;
        w[0] = 1.0f - f;
        w[1] = f;
    } else {
        w[0] = 1.0f;
        w[1] = 0.0f;
    }
}

constexpr int kMaxApplyThreads = 256;

// Asynchronous 4-byte copy global -> shared; with ok == false nothing is read
// and the destination is filled with zero (src only has to be a valid address).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}
constexpr int kApplyVectors = 4;   // vectors per CTA (they share the staged PSFs)

// The correlations of 4 consecutive outputs of one row with the cell's NC PSFs:
// acc[c][o] = sum_{dz, dx} p_c(dz, dx) v(row + dz, col + o + dx), from the patch
// rows starting at `vrow` (pitch PWX floats, the strip's float4 column s) and
// the PSFs at `sp` (NC of [W][W4]).
template <int NC>
__device__ __forceinline__ void correlate_strip(const float *__restrict__ vrow, int PWX, int s,
                                                const float *__restrict__ sp, int W, int W4, float (&acc)[4][4])
{
    const int cstride = W * W4 / 4;   // float4s per PSF
    for (int dz = 0; dz < W; ++dz) {
        const float4 *vr = reinterpret_cast<const float4 *>(vrow + dz * PWX) + s;
        const float4 *pr = reinterpret_cast<const float4 *>(sp + dz * W4);
        float4 cur = vr[0];
#pragma unroll 2
        for (int d4 = 0; d4 < W4 / 4; ++d4) {
            const float4 nxt = vr[d4 + 1];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float4 p = pr[c * cstride + d4];
                acc[c][0] = fmaf(p.w, cur.w, fmaf(p.z, cur.z, fmaf(p.y, cur.y, fmaf(p.x, cur.x, acc[c][0]))));
                acc[c][1] = fmaf(p.w, nxt.x, fmaf(p.z, cur.w, fmaf(p.y, cur.z, fmaf(p.x, cur.y, acc[c][1]))));
                acc[c][2] = fmaf(p.w, nxt.y, fmaf(p.z, nxt.x, fmaf(p.y, cur.w, fmaf(p.x, cur.z, acc[c][2]))));
                acc[c][3] = fmaf(p.w, nxt.z, fmaf(p.z, nxt.y, fmaf(p.y, nxt.x, fmaf(p.x, cur.w, acc[c][3]))));
            }
            cur = nxt;
        }
    }
}

// out_j(x) = sum over the cell's lattice points k of w_k(x) (p_k correlated with v_j)(x).
// grid = (cells along x, cells along z, groups of 4 vectors).  The CTA stages
// the cell's 1, 2 or 4 PSFs (rows zero-padded to a multiple of 4) and, per
// vector, the patch of v_j the cell's correlations read (zero off the grid) in
// shared memory; each thread computes 4 consecutive outputs of a row of one
// vector against all of the cell's PSFs, so one float4 of v feeds 16
// multiply-adds per PSF.
__global__ void __launch_bounds__(kMaxApplyThreads) k_psf_apply(const float *__restrict__ psf,
                                                                 const float *__restrict__ v,
                                                                 float *__restrict__ out, PsfGeo g)
{
    extern __shared__ float4 sm4[];
    const CellAxis az = cell_axis(blockIdx.y, g.cz0, g.S, g.na, g.nz);
    const CellAxis ax = cell_axis(blockIdx.x, g.cx0, g.S, g.nb, g.nx);
    if (az.lo >= az.hi || ax.lo >= ax.hi) return;       // empty edge cell (first point on the edge)
    const int j0 = blockIdx.z * g.vpc, nvec = min(g.vpc, g.k - j0);
    const int R = g.R, W = 2 * R + 1, W4 = (W + 3) & ~3;
    const int rows = az.hi - az.lo, nstrip = (ax.hi - ax.lo + 3) / 4;
    const int PWX = 4 * nstrip + W4 + 4, PH = rows + 2 * R;
    const int nc = az.np * ax.np;
    float *sp = reinterpret_cast<float *>(sm4);         // [nc][W][W4]
    float *sv = sp + 4 * W * W4;                        // [nvec][PH][PWX]
    // Every staged element is one independent asynchronous copy, so the CTA
    // waits for one memory latency, not one per row.
    for (int i = threadIdx.x; i < nc * W * W4; i += blockDim.x) {
        const int c = i / (W * W4), r = i - c * (W * W4);
        const int dz = r / W4, dx = r - dz * W4;
        const int k = (az.p0 + c / ax.np) * g.nb + ax.p0 + c % ax.np;
        cp_async4(sp + i, dx < W ? psf + ((size_t)k * W + dz) * W + dx : psf, dx < W);
    }
    for (int i = threadIdx.x; i < nvec * PH * PWX; i += blockDim.x) {
        const int q = i / (PH * PWX), r = i - q * (PH * PWX);
        const int z = az.lo - R + r / PWX, x = ax.lo - R + r % PWX;
        const bool in = z >= 0 && z < g.nz && x >= 0 && x < g.nx;
        const float *vj = v + (size_t)(j0 + q) * g.nz * g.nx;
        cp_async4(sv + i, in ? vj + (size_t)z * g.nx + x : vj, in);
    }
    cp_async_wait_all();
    __syncthreads();
    const int per_vec = rows * nstrip;
    for (int it = threadIdx.x; it < nvec * per_vec; it += blockDim.x) {
        const int q = it / per_vec, rs = it - q * per_vec;
        const int r = rs / nstrip, s = rs - r * nstrip;
        const int j = j0 + q;
        float acc[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[c][o] = 0.0f;
        const float *vrow = sv + (q * PH + r) * PWX;
        if (nc == 4) correlate_strip<4>(vrow, PWX, s, sp, W, W4, acc);
        else if (nc == 2) correlate_strip<2>(vrow, PWX, s, sp, W, W4, acc);
        else correlate_strip<1>(vrow, PWX, s, sp, W, W4, acc);
        const int iz = az.lo + r;
        float wz[2];
        cell_weights(az, iz, g.S, wz);
        float *orow = out + (size_t)j * g.nz * g.nx + (size_t)iz * g.nx;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int ix = ax.lo + 4 * s + o;
            if (ix < ax.hi) {
                float wx[2];
                cell_weights(ax, ix, g.S, wx);
                float y = 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool zi = c / ax.np != 0, xi = c % ax.np != 0;   // which of the cell's points
                    if (c < nc) y = fmaf((zi ? wz[1] : wz[0]) * (xi ? wx[1] : wx[0]), acc[c][o], y);
                }
                orow[ix] = y;
            }
        }
    }
}

int check_launch(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

}  // namespace

int psf_apply_smem_bytes(int S, int R, int nvec)
{
    const int W = 2 * R + 1, W4 = (W + 3) & ~3;
    const int rows = S, nstrip = (S + 3) / 4;   // the largest cell is S x S
    return (nvec * (rows + 2 * R) * (4 * nstrip + W4 + 4) + 4 * W * W4) * (int)sizeof(float);
}

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
    PsfGeo gk = g;
    gk.k = k;
    int nvec = kApplyVectors;   // fewer vectors per CTA when their patches would not fit
    while (nvec > 1 && psf_apply_smem_bytes(g.S, g.R, nvec) > 200 * 1024) --nvec;
    const int smem = psf_apply_smem_bytes(g.S, g.R, nvec);
    static std::mutex mu;
    static int granted[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return hvi::fail(HV_EINVAL, "internal: device %d", dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (smem > granted[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_psf_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess)
                return hvi::fail(HV_ECUDA, "PSF apply needs %d bytes of shared memory: %s", smem, cudaGetErrorString(e));
            granted[dev] = smem;
        }
    }
    const int items = std::min(nvec, k) * g.S * ((g.S + 3) / 4);   // 4-point strips of the largest cell
    const int threads = std::min(kMaxApplyThreads, (items + 31) / 32 * 32);
    dim3 grid(g.nb + 1, g.na + 1, (k + nvec - 1) / nvec);
    gk.vpc = nvec;
    k_psf_apply<<<grid, threads, smem, st>>>(psf, v, out, gk);
    return check_launch("k_psf_apply");
}

}  // namespace hvk
