// hv_kernels.cu -- sm_103a kernels of the Gauss-Newton Hessian apply.
//
// Discrete operator (section 2, eq. (pde), with a damping-rate sponge): with
// C = m^2 dt^2 / h^2, a = q dt / 2 and the unscaled 8th-order stencil sum
//   Lh w = 2 c0 w + sum_{k=1..4} c_k (w[x-k] + w[x+k] + w[z-k] + w[z+k]),
//   c0 = -205/72, c1 = 8/5, c2 = -1/5, c3 = 8/315, c4 = -1/560
// one leapfrog row reads
//   (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} + C (Lh u^n + s_n delta_src)
// (the source s_n/h^2 times m^2 dt^2 is C s_n).  Because S depends on m only
// through 1/m^2, the Born source is (2 dm / m^3) (T u)^n = (2 dm / m)(L u^n + f^n):
//   (1 + a) du^{n+1} = 2 du^n - (1 - a) du^{n-1} + C (Lh du^n + b Q^n),
//   b = 2 dm / m, Q^n = Lh u^n + s_n delta_src,
// the adjoint is the same stepper run backward with receiver sources,
//   (1 + a) lam^n = 2 lam^{n+1} - (1 - a) lam^{n+2} + C (Lh lam^{n+1} + h^2 g^n),
// and the zero-lag image is G^T lam = (2 / (m h^2)) sum_n lam^n Q^n, accumulated
// here as sum_n lam^n Q^n in FP64 and scaled at the end.  No step forms the
// three-level difference u^{n+1} - 2u^n + u^{n-1}, so FP32 loses nothing to
// cancellation.
//
// All stencil kernels share one engine: a CTA owns a TX x TZ tile, stages the
// tile plus its 4-cell halo in shared memory with coalesced float4 loads
// (the ghost band makes every load unconditional inside the allocation), and
// each thread computes a 4 (x) x RZ (z) register block from shared memory.
#include "hv_internal.h"

#include <atomic>
#include <cmath>

namespace hvk {

using hvi::GH;

namespace {

constexpr float LC1 = (float)(8.0 / 5.0);
constexpr float LC2 = (float)(-1.0 / 5.0);
constexpr float LC3 = (float)(8.0 / 315.0);
constexpr float LC4 = (float)(-1.0 / 560.0);

// Stencil tile configuration: BX x BZ threads, each 4 x RZ points.
template <int BX_, int BZ_, int RZ_>
struct Cfg {
    static constexpr int BX = BX_, BZ = BZ_, RZ = RZ_;
    static constexpr int NT = BX * BZ;
    static constexpr int TX = 4 * BX, TZ = RZ * BZ;
    static constexpr int W = TX + 2 * GH, H = TZ + 2 * GH;
    static constexpr int W4 = W / 4;
};

using CfgF = Cfg<16, 16, 2>;   // forward / Born / recompute: 64 x 32 tiles
using CfgA = Cfg<16, 16, 2>;   // adjoint + imaging: 64 x 32 tiles

struct Geo {
    int P, rows, NZ, NX, ntx;
    size_t fsize;
};

__device__ __forceinline__ Geo geo_of(int P, int rows, int NZ, int NX, int ntx, size_t fsize)
{
    return Geo{P, rows, NZ, NX, ntx, fsize};
}

// Stage allocation rows z0 .. z0+H-1, columns x0 .. x0+W-1 (z0, x0 = padded tile
// origin, which is the allocation origin of its halo) into sm[H][W].
template <class C>
__device__ __forceinline__ void load_tile(float *__restrict__ sm, const float *__restrict__ g, const Geo &G,
                                          int z0, int x0)
{
    float4 *s4 = reinterpret_cast<float4 *>(sm);
    for (int idx = threadIdx.x; idx < C::H * C::W4; idx += C::NT) {
        int i = idx / C::W4;
        int q = idx - i * C::W4;
        int gz = z0 + i, gx = x0 + 4 * q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gz < G.rows && gx < G.P) v = __ldg(reinterpret_cast<const float4 *>(g + (size_t)gz * G.P + gx));
        s4[idx] = v;
    }
}

__device__ __forceinline__ float comp(const float4 &v, int c)
{
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Lh at the thread's 4 x RZ block; also returns the centre values.  The sum is
// taken over differences from the centre, sum_k c_k ((w[+k] - w0) + (w[-k] - w0)),
// which equals Lh w because c0 + 2 sum_k c_k = 0; for smooth fields each
// difference is small and nearly exact in FP32, so the rounding error of Lh
// scales with |Lh w| rather than with |w| (about 7x lower wavefield error
// after 600 steps than the direct sum, at no extra memory traffic).
template <class C>
__device__ __forceinline__ void lap_block(const float *__restrict__ sm, int tx, int tz, float (&L)[C::RZ][4],
                                          float (&ctr)[C::RZ][4])
{
    const float4 *s4 = reinterpret_cast<const float4 *>(sm);
    float4 col[C::RZ + 8];
#pragma unroll
    for (int i = 0; i < C::RZ + 8; ++i) col[i] = s4[(tz * C::RZ + i) * C::W4 + tx + 1];
#pragma unroll
    for (int r = 0; r < C::RZ; ++r) {
        const int row = tz * C::RZ + r + GH;
        float4 xm = s4[row * C::W4 + tx];
        float4 xc = col[r + 4];
        float4 xp = s4[row * C::W4 + tx + 2];
        float v[12] = {xm.x, xm.y, xm.z, xm.w, xc.x, xc.y, xc.z, xc.w, xp.x, xp.y, xp.z, xp.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float cz = v[4 + c];
            auto pair = [cz](float a, float b) { return (a - cz) + (b - cz); };
            float acc = LC4 * (pair(v[c], v[8 + c]) + pair(comp(col[r], c), comp(col[r + 8], c)));
            acc = fmaf(LC3, pair(v[1 + c], v[7 + c]) + pair(comp(col[r + 1], c), comp(col[r + 7], c)), acc);
            acc = fmaf(LC2, pair(v[2 + c], v[6 + c]) + pair(comp(col[r + 2], c), comp(col[r + 6], c)), acc);
            acc = fmaf(LC1, pair(v[3 + c], v[5 + c]) + pair(comp(col[r + 3], c), comp(col[r + 5], c)), acc);
            L[r][c] = acc;
            ctr[r][c] = cz;
        }
    }
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// Store 4 consecutive x values at padded (z, x..x+3), skipping x >= NX.
__device__ __forceinline__ void st4(float *p, float4 v, int x, int NX)
{
    if (x + 3 < NX) {
        *reinterpret_cast<float4 *>(p) = v;
    } else {
        if (x + 0 < NX) p[0] = v.x;
        if (x + 1 < NX) p[1] = v.y;
        if (x + 2 < NX) p[2] = v.z;
        if (x + 3 < NX) p[3] = v.w;
    }
}

struct FwdParams {
    const float *u_cur, *u_prev;
    float *u_next;
    const float *C, *b, *az, *ax, *wavelet;
    const float *du_cur;
    float *du_io;
    float *d_u, *d_du;
    const int *src_zx;
    const int *rt_off, *rt_rec, *rt_pos;
    int n, nt, nr, ns, k, vpg;
    int P, rows, NZ, NX, ntx, ntiles;
    size_t fsize;
};

// One forward time step for one (tile, shot, vector group):
//   u^{n+1} (group 0 only) and du_j^{n+1} for the group's vectors, with fused
//   receiver sampling.  grid = (ntiles, ns, ngroups).
template <class C, bool BORN>
__global__ void __launch_bounds__(C::NT) k_fwd(const __grid_constant__ FwdParams p)
{
    __shared__ __align__(16) float su[C::H * C::W];
    __shared__ __align__(16) float sd[BORN ? C::H * C::W : 4];
    const Geo G = geo_of(p.P, p.rows, p.NZ, p.NX, p.ntx, p.fsize);
    const int tile = blockIdx.x, s = blockIdx.y, grp = blockIdx.z;
    const int tzi = tile / p.ntx, txi = tile - tzi * p.ntx;
    const int z0 = tzi * C::TZ, x0 = txi * C::TX;          // padded tile origin
    const int tx = threadIdx.x % C::BX, tz = threadIdx.x / C::BX;
    const size_t so = (size_t)s * p.fsize;

    load_tile<C>(su, p.u_cur + so, G, z0, x0);
    __syncthreads();

    float Q[C::RZ][4], uc[C::RZ][4];
    lap_block<C>(su, tx, tz, Q, uc);
    const int sz = p.src_zx[2 * s], sx = p.src_zx[2 * s + 1];
    const float wav = p.wavelet[p.n];
    const int xb = x0 + 4 * tx;                            // padded x of component 0
    float axv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) axv[c] = p.ax[min(xb + c, p.NX - 1)];
    float Cc[C::RZ][4], inv[C::RZ][4], oma[C::RZ][4];
#pragma unroll
    for (int r = 0; r < C::RZ; ++r) {
        const int z = z0 + tz * C::RZ + r;
        const float azv = p.az[min(z, p.NZ - 1)];
        const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
        float4 c4 = (z < p.NZ && xb < p.NX) ? ldg4(p.C + off) : make_float4(0.f, 0.f, 0.f, 0.f);
        Cc[r][0] = c4.x; Cc[r][1] = c4.y; Cc[r][2] = c4.z; Cc[r][3] = c4.w;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (z == sz && xb + c == sx) Q[r][c] += wav;
            float a = fmaxf(azv, axv[c]);
            inv[r][c] = __frcp_rn(1.0f + a);
            oma[r][c] = 1.0f - a;
        }
    }

    const int tb = s * (p.ntiles + 1) + tile;
    const int rb = p.rt_off[tb], re = p.rt_off[tb + 1];

    if (grp == 0 && p.u_next) {
        float *un = p.u_next + so;
#pragma unroll
        for (int r = 0; r < C::RZ; ++r) {
            const int z = z0 + tz * C::RZ + r;
            if (z >= p.NZ || xb >= p.NX) continue;
            const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
            float4 pv = ldg4(p.u_prev + so + off);
            float pr[4] = {pv.x, pv.y, pv.z, pv.w};
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                o[c] = inv[r][c] * (2.0f * uc[r][c] - oma[r][c] * pr[c] + Cc[r][c] * Q[r][c]);
            st4(un + off, make_float4(o[0], o[1], o[2], o[3]), xb, p.NX);
        }
        if (p.d_u && rb < re) {
            __syncthreads();
            for (int i = rb + threadIdx.x; i < re; i += C::NT)
                p.d_u[((size_t)s * p.nt + p.n) * p.nr + p.rt_rec[s * p.nr + i]] = un[p.rt_pos[s * p.nr + i]];
        }
    }

    if constexpr (BORN) {
        const int j0 = grp * p.vpg, j1 = min(p.k, j0 + p.vpg);
        for (int j = j0; j < j1; ++j) {
            const size_t fo = ((size_t)j * p.ns + s) * p.fsize;
            __syncthreads();                       // sd reuse across vectors
            load_tile<C>(sd, p.du_cur + fo, G, z0, x0);
            __syncthreads();
            float Ld[C::RZ][4], dc[C::RZ][4];
            lap_block<C>(sd, tx, tz, Ld, dc);
            float *dn = p.du_io + fo;
#pragma unroll
            for (int r = 0; r < C::RZ; ++r) {
                const int z = z0 + tz * C::RZ + r;
                if (z >= p.NZ || xb >= p.NX) continue;
                const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
                float4 pv = ld4(dn + off);
                float4 bv = ldg4(p.b + (size_t)j * p.fsize + off);
                float pr[4] = {pv.x, pv.y, pv.z, pv.w};
                float bb[4] = {bv.x, bv.y, bv.z, bv.w};
                float o[4];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    o[c] = inv[r][c] *
                           (2.0f * dc[r][c] - oma[r][c] * pr[c] + Cc[r][c] * (Ld[r][c] + bb[c] * Q[r][c]));
                st4(dn + off, make_float4(o[0], o[1], o[2], o[3]), xb, p.NX);
            }
            if (p.d_du && rb < re) {
                __syncthreads();
                for (int i = rb + threadIdx.x; i < re; i += C::NT)
                    p.d_du[(((size_t)j * p.ns + s) * p.nt + p.n) * p.nr + p.rt_rec[s * p.nr + i]] =
                        dn[p.rt_pos[s * p.nr + i]];
            }
        }
    }
}

struct AdjParams {
    const float *u, *lam1;
    float *lam_io;
    const float *C, *az, *ax, *wavelet;
    const float *r;
    size_t r_vstride;
    float rscale;
    double *img;
    const int *src_zx;
    const int *rt_off, *rt_rec, *rt_pos;
    int n, nt, nr, ns, k, spg;
    int P, rows, NZ, NX, ntx, ntiles;
    size_t fsize;
};

// One adjoint time step with zero-lag imaging for one (tile, vector, shot
// group); the CTA loops over its shots in order and adds its FP64 image
// contribution once.  grid = (ntiles, k, G).
template <class C>
__global__ void __launch_bounds__(C::NT) k_adj(const __grid_constant__ AdjParams p)
{
    __shared__ __align__(16) float su[C::H * C::W];
    __shared__ __align__(16) float sl[C::H * C::W];
    __shared__ __align__(16) float ssrc[C::TZ * C::TX];
    const Geo G = geo_of(p.P, p.rows, p.NZ, p.NX, p.ntx, p.fsize);
    const int tile = blockIdx.x, j = blockIdx.y, g = blockIdx.z;
    const int tzi = tile / p.ntx, txi = tile - tzi * p.ntx;
    const int z0 = tzi * C::TZ, x0 = txi * C::TX;
    const int tx = threadIdx.x % C::BX, tz = threadIdx.x / C::BX;
    const int xb = x0 + 4 * tx;
    const float wav = p.wavelet[p.n];

    float axv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) axv[c] = p.ax[min(xb + c, p.NX - 1)];
    float Cc[C::RZ][4], inv[C::RZ][4], oma[C::RZ][4];
#pragma unroll
    for (int r = 0; r < C::RZ; ++r) {
        const int z = z0 + tz * C::RZ + r;
        const float azv = p.az[min(z, p.NZ - 1)];
        const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
        float4 c4 = (z < p.NZ && xb < p.NX) ? ldg4(p.C + off) : make_float4(0.f, 0.f, 0.f, 0.f);
        Cc[r][0] = c4.x; Cc[r][1] = c4.y; Cc[r][2] = c4.z; Cc[r][3] = c4.w;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float a = fmaxf(azv, axv[c]);
            inv[r][c] = __frcp_rn(1.0f + a);
            oma[r][c] = 1.0f - a;
        }
    }
    double acc[C::RZ][4];
#pragma unroll
    for (int r = 0; r < C::RZ; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    const int s0 = g * p.spg, s1 = min(p.ns, s0 + p.spg);
    for (int s = s0; s < s1; ++s) {
        const size_t so = (size_t)s * p.fsize;
        const size_t fo = ((size_t)j * p.ns + s) * p.fsize;
        const int tb = s * (p.ntiles + 1) + tile;
        const int rb = p.rt_off[tb], re = p.rt_off[tb + 1];
        __syncthreads();                           // smem reuse across shots
        load_tile<C>(su, p.u + so, G, z0, x0);
        load_tile<C>(sl, p.lam1 + fo, G, z0, x0);
        if (rb < re) {
            for (int i = threadIdx.x; i < C::TZ * C::TX; i += C::NT) ssrc[i] = 0.0f;
            __syncthreads();
            const float *rs = p.r + (size_t)j * p.r_vstride + ((size_t)s * p.nt + p.n) * p.nr;
            for (int i = rb + threadIdx.x; i < re; i += C::NT) {
                int pos = p.rt_pos[s * p.nr + i];
                int zz = pos / p.P - GH - z0, xx = pos % p.P - GH - x0;
                ssrc[zz * C::TX + xx] = p.rscale * rs[p.rt_rec[s * p.nr + i]];
            }
        }
        __syncthreads();
        float Qu[C::RZ][4], ucen[C::RZ][4], Ll[C::RZ][4], lc[C::RZ][4];
        lap_block<C>(su, tx, tz, Qu, ucen);
        lap_block<C>(sl, tx, tz, Ll, lc);
        const int sz = p.src_zx[2 * s], sx = p.src_zx[2 * s + 1];
        float *ln = p.lam_io + fo;
#pragma unroll
        for (int r = 0; r < C::RZ; ++r) {
            const int z = z0 + tz * C::RZ + r;
            const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
            float src[4] = {0.f, 0.f, 0.f, 0.f};
            if (rb < re) {
                float4 sv = *reinterpret_cast<const float4 *>(&ssrc[(tz * C::RZ + r) * C::TX + 4 * tx]);
                src[0] = sv.x; src[1] = sv.y; src[2] = sv.z; src[3] = sv.w;
            }
            if (z >= p.NZ || xb >= p.NX) continue;
            float4 pv = ld4(ln + off);
            float pr[4] = {pv.x, pv.y, pv.z, pv.w};
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float q = Qu[r][c];
                if (z == sz && xb + c == sx) q += wav;
                o[c] = inv[r][c] * (2.0f * lc[r][c] - oma[r][c] * pr[c] + Cc[r][c] * (Ll[r][c] + src[c]));
                acc[r][c] += (double)o[c] * (double)q;
            }
            st4(ln + off, make_float4(o[0], o[1], o[2], o[3]), xb, p.NX);
        }
    }
    double *im = p.img + ((size_t)g * p.k + j) * p.fsize;
#pragma unroll
    for (int r = 0; r < C::RZ; ++r) {
        const int z = z0 + tz * C::RZ + r;
        if (z >= p.NZ || xb >= p.NX) continue;
        const size_t off = (size_t)(z + GH) * p.P + (xb + GH);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (xb + c < p.NX) im[off + c] += acc[r][c];
    }
}

// m (interior) -> C on the padded grid; v_j -> b_j = 2 (E v_j) / (E m).
__global__ void k_prep(const float *__restrict__ m, const float *__restrict__ v, int k, float *__restrict__ Cc,
                       float *__restrict__ b, int nz, int nx, int nb, int NZ, int NX, int P, size_t fsize, double dt,
                       double h)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (x >= NX || z >= NZ) return;
    const int iz = min(max(z - nb, 0), nz - 1), ix = min(max(x - nb, 0), nx - 1);
    const double mm = (double)m[(size_t)iz * nx + ix];
    const size_t off = (size_t)(z + GH) * P + (x + GH);
    const double cdt = mm * dt / h;
    Cc[off] = (float)(cdt * cdt);
    if (b)
        for (int j = 0; j < k; ++j)
            b[(size_t)j * fsize + off] = (float)(2.0 * (double)v[((size_t)j * nz + iz) * nx + ix] / mm);
}

// Hv[j][iz][ix] = (2 / (m h^2)) sum over the E-preimage of (iz, ix) of sum_g img[g][j].
__global__ void k_finalize(const float *__restrict__ m, const double *__restrict__ img, int G, int k, int nz, int nx,
                           int nb, int NZ, int NX, int P, size_t fsize, double h, float *out32, double *out64)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int j = blockIdx.z;
    if (ix >= nx) return;
    const int zlo = (iz == 0) ? 0 : iz + nb, zhi = (iz == nz - 1) ? NZ - 1 : iz + nb;
    const int xlo = (ix == 0) ? 0 : ix + nb, xhi = (ix == nx - 1) ? NX - 1 : ix + nb;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z)
        for (int x = xlo; x <= xhi; ++x) {
            const size_t off = (size_t)(z + GH) * P + (x + GH);
            for (int g = 0; g < G; ++g) acc += img[((size_t)g * k + j) * fsize + off];
        }
    const double mm = (double)m[(size_t)iz * nx + ix];
    const double val = 2.0 / (mm * h * h) * acc;
    const size_t o = ((size_t)j * nz + iz) * nx + ix;
    if (out32) out32[o] = (float)val;
    if (out64) out64[o] = val;
}

// r = d - dobs and per-block FP64 partial sums of r^2 (fixed assignment, fixed tree).
__global__ void k_residual(const float *d, const float *__restrict__ dobs, float *r,
                           size_t n, double *__restrict__ partials)
{
    __shared__ double sw[32];
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double e = (double)d[i] - (double)dobs[i];
        r[i] = (float)e;
        acc += e * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void k_reduce_phi(const double *__restrict__ partials, int nb, double scale, double *phi)
{
    __shared__ double sw[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *phi = scale * v;
    }
}

// Zero the ghost band (the Dirichlet zeros every stencil read relies on) of
// nfields consecutive fields: rows [0, 4) and [NZ+4, rows), and columns
// [0, 4) and [NX+4, P) of the other rows.  Workspace memory arrives
// uninitialised; the kernels never write the band, so this runs once per call.
__global__ void k_zero_ghosts(float *__restrict__ f, long long nfields, int NZ, int NX, int P, int rows, size_t fsize)
{
    const int per_row_side = P - NX;                    // ghost columns per interior row
    const long long per_field = (long long)2 * GH * P + (long long)NZ * per_row_side;
    const long long total = per_field * nfields;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long fld = i / per_field;
        long long r = i - fld * per_field;
        size_t off;
        if (r < (long long)GH * P) {
            off = (size_t)r;                                          // top ghost rows
        } else if (r < (long long)2 * GH * P) {
            off = (size_t)(NZ + GH) * P + (size_t)(r - (long long)GH * P);   // bottom ghost rows
        } else {
            r -= (long long)2 * GH * P;
            const int z = (int)(r / per_row_side), c = (int)(r - (long long)z * per_row_side);
            const int x = (c < GH) ? c : NX + c;                      // left band, then right band
            off = (size_t)(z + GH) * P + x;
        }
        f[(size_t)fld * fsize + off] = 0.0f;
    }
    (void)rows;
}

// Padded-grid copy of a field batch out of the ghost layout: out[s][NZ][NX].
__global__ void k_copy_wavefield(const float *__restrict__ u, float *__restrict__ out, int NZ, int NX, int P,
                                 size_t fsize)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y, s = blockIdx.z;
    if (x >= NX) return;
    out[((size_t)s * NZ + z) * NX + x] = u[(size_t)s * fsize + (size_t)(z + GH) * P + (x + GH)];
}

// Source wavelet and sponge profiles (a = q dt / 2 per axis), computed once per handle.
__global__ void k_setup(float *wavelet, int nt, double dt, double f0, double t0, float *az, int NZ, float *ax,
                        int NX, int nb, int nz, int nx, double h, double qmax)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) {
        const double tau = i * dt - t0;
        const double a = M_PI * M_PI * f0 * f0 * tau * tau;
        wavelet[i] = (float)((1.0 - 2.0 * a) * exp(-a));
    }
    const double L = nb * h;
    if (i < NZ) {
        double d = 0.0;
        if (i < nb) d = (nb - i) * h;
        else if (i >= nb + nz) d = (i - (nb + nz) + 1) * h;
        az[i] = (nb > 0) ? (float)(0.5 * dt * qmax * (d / L) * (d / L)) : 0.0f;
    }
    if (i < NX) {
        double d = 0.0;
        if (i < nb) d = (nb - i) * h;
        else if (i >= nb + nx) d = (i - (nb + nx) + 1) * h;
        ax[i] = (nb > 0) ? (float)(0.5 * dt * qmax * (d / L) * (d / L)) : 0.0f;
    }
}

int cuda_check(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

template <class C>
hvi::Tiling make_tiling(const hv_handle *h)
{
    hvi::Tiling t;
    t.TX = C::TX;
    t.TZ = C::TZ;
    t.ntx = (h->NX + C::TX - 1) / C::TX;
    t.ntz = (h->NZ + C::TZ - 1) / C::TZ;
    t.ntiles = t.ntx * t.ntz;
    return t;
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

hvi::Tiling tiling_fwd(const hv_handle *h) { return make_tiling<CfgF>(h); }
hvi::Tiling tiling_adj(const hv_handle *h) { return make_tiling<CfgA>(h); }

// Shot groups of the adjoint kernel.  Each group sums its shots' image
// contributions in shot order into its own FP64 partial image; the groups are
// summed in group order at the end.  The count depends only on the grid and
// the shot count (never on k), so a vector's result is bitwise the same
// whether it is applied alone or in a batch.
int adj_groups(const hv_handle *h)
{
    hvi::Tiling t = tiling_adj(h);
    long long ctas = (long long)t.ntiles;
    int G = (int)((608 + ctas - 1) / ctas);
    if (G < 1) G = 1;
    if (G > h->ns) G = h->ns;
    int spg = (h->ns + G - 1) / G;
    return (h->ns + spg - 1) / spg;
}

int launch_fwd(const hv_handle *h, const hvi::RecTiles &rt, const FwdLaunch &a, cudaStream_t st)
{
    hvi::Tiling t = tiling_fwd(h);
    FwdParams p{};
    p.u_cur = a.u_cur; p.u_prev = a.u_prev; p.u_next = a.u_next;
    p.C = a.C; p.b = a.b; p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
    p.du_cur = a.du_cur; p.du_io = a.du_io; p.d_u = a.d_u; p.d_du = a.d_du;
    p.src_zx = h->src_zx; p.rt_off = rt.off; p.rt_rec = rt.rec; p.rt_pos = rt.pos;
    p.n = a.n; p.nt = h->nt; p.nr = h->nr; p.ns = h->ns; p.k = a.k;
    p.P = h->P; p.rows = h->rows; p.NZ = h->NZ; p.NX = h->NX; p.ntx = t.ntx; p.ntiles = t.ntiles;
    p.fsize = h->fsize;
    const bool born = a.b != nullptr && a.k > 0;
    int groups = 1;
    if (born) {
        // enough CTAs to fill the machine; each group recomputes Q from u
        long long base = (long long)t.ntiles * h->ns;
        groups = (int)((608 + base - 1) / base);
        if (groups > a.k) groups = a.k;
        if (groups < 1) groups = 1;
        p.vpg = (a.k + groups - 1) / groups;
        groups = (a.k + p.vpg - 1) / p.vpg;
    } else {
        p.vpg = 0;
    }
    dim3 grid(t.ntiles, h->ns, groups);
    if (born) k_fwd<CfgF, true><<<grid, CfgF::NT, 0, st>>>(p);
    else k_fwd<CfgF, false><<<grid, CfgF::NT, 0, st>>>(p);
    return cuda_check("k_fwd launch");
}

int launch_adj(const hv_handle *h, const hvi::RecTiles &rt, const AdjLaunch &a, cudaStream_t st)
{
    hvi::Tiling t = tiling_adj(h);
    AdjParams p{};
    p.u = a.u; p.lam1 = a.lam1; p.lam_io = a.lam_io;
    p.C = a.C; p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
    p.r = a.r; p.r_vstride = a.r_per_vector ? (size_t)h->ns * h->nt * h->nr : 0; p.rscale = a.rscale;
    p.img = a.img; p.src_zx = h->src_zx; p.rt_off = rt.off; p.rt_rec = rt.rec; p.rt_pos = rt.pos;
    p.n = a.n; p.nt = h->nt; p.nr = h->nr; p.ns = h->ns; p.k = a.k;
    p.spg = (h->ns + a.G - 1) / a.G;
    p.P = h->P; p.rows = h->rows; p.NZ = h->NZ; p.NX = h->NX; p.ntx = t.ntx; p.ntiles = t.ntiles;
    p.fsize = h->fsize;
    dim3 grid(t.ntiles, a.k, a.G);
    k_adj<CfgA><<<grid, CfgA::NT, 0, st>>>(p);
    return cuda_check("k_adj launch");
}

int launch_prep(const hv_handle *h, const float *m, const float *v, int k, float *C, float *b, cudaStream_t st)
{
    dim3 grid((h->NX + 127) / 128, h->NZ);
    k_prep<<<grid, 128, 0, st>>>(m, v, k, C, b, h->nz, h->nx, h->nb, h->NZ, h->NX, h->P, h->fsize, h->dt, h->h);
    return cuda_check("k_prep launch");
}

int launch_finalize(const hv_handle *h, const float *m, const double *img, int G, int k, float *out32,
                    double *out64, cudaStream_t st)
{
    dim3 grid((h->nx + 127) / 128, h->nz, k);
    k_finalize<<<grid, 128, 0, st>>>(m, img, G, k, h->nz, h->nx, h->nb, h->NZ, h->NX, h->P, h->fsize, h->h, out32,
                                     out64);
    return cuda_check("k_finalize launch");
}

int launch_residual(const hv_handle *h, const float *d, const float *dobs, float *r, double *partials, int nblocks,
                    cudaStream_t st)
{
    size_t n = (size_t)h->ns * h->nt * h->nr;
    k_residual<<<nblocks, 256, 0, st>>>(d, dobs, r, n, partials);
    return cuda_check("k_residual launch");
}

int launch_reduce_phi(const double *partials, int nblocks, double scale, double *phi, cudaStream_t st)
{
    k_reduce_phi<<<1, 1024, 0, st>>>(partials, nblocks, scale, phi);
    return cuda_check("k_reduce_phi launch");
}

int launch_zero_ghosts(const hv_handle *h, float *f, long long nfields, cudaStream_t st)
{
    if (nfields <= 0) return HV_OK;
    long long per_field = (long long)2 * GH * h->P + (long long)h->NZ * (h->P - h->NX);
    long long total = per_field * nfields;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    k_zero_ghosts<<<(unsigned)blocks, 256, 0, st>>>(f, nfields, h->NZ, h->NX, h->P, h->rows, h->fsize);
    return cuda_check("k_zero_ghosts launch");
}

int launch_copy_wavefield(const hv_handle *h, const float *u, float *out, cudaStream_t st)
{
    dim3 grid((h->NX + 127) / 128, h->NZ, h->ns);
    k_copy_wavefield<<<grid, 128, 0, st>>>(u, out, h->NZ, h->NX, h->P, h->fsize);
    return cuda_check("k_copy_wavefield launch");
}

int launch_setup(hv_handle *h, cudaStream_t st)
{
    int n = h->nt;
    if (h->NZ > n) n = h->NZ;
    if (h->NX > n) n = h->NX;
    double L = h->nb * h->h;
    double qmax = (h->nb > 0) ? 3.0 * h->vmax * std::log(1.0 / h->R) / (2.0 * L) : 0.0;
    k_setup<<<(n + 127) / 128, 128, 0, st>>>(h->wavelet, h->nt, h->dt, h->f0, h->t0, h->az, h->NZ, h->ax, h->NX,
                                             h->nb, h->nz, h->nx, h->h, qmax);
    return cuda_check("k_setup launch");
}

}  // namespace hvk
