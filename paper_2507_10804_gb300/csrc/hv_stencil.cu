// hv_stencil.cu -- the time-stepping kernels (forward / Born / recompute and
// adjoint + imaging) on sm_103a: TMA-staged shared-memory tiles pipelined
// across shots.
//
// Operator (section 2, eq. (pde) with the damping-rate sponge; C = (m dt/h)^2,
// a = q dt / 2, Lh = h^2 L the unscaled 8th-order sum, s_n the source):
//   (1 + a) u^{n+1}   = 2 u^n - (1 - a) u^{n-1} + C (Lh u^n + s_n delta_src)
//   (1 + a) du^{n+1}  = 2 du^n - (1 - a) du^{n-1} + C (Lh du^n + b Q^n),  b = 2 dm / m
//   (1 + a) lam^n     = 2 lam^{n+1} - (1 - a) lam^{n+2} + C (Lh lam^{n+1} + h^2 g^n)
//   image            += lam^n Q^n,  Q^n = Lh u^n + s_n delta_src
//                       (per step: FP32 over <= 8 shots, then added to a double-float image)
// The Born source and the image use (T u)^n = m^2 (L u^n + f^n), the exact
// identity of the forward rows, so no FP32 step forms u^{n+1} - 2u^n + u^{n-1}.
//
// Work decomposition: a CTA owns one TX x TZ tile of the padded grid, one
// vector j and a group of up to 8 shots, and walks its shots in order.  The
// whole workspace is one 3D tensor (x, z, field index) for the Tensor Memory
// Accelerator: for each shot one thread issues bulk tile copies of the
// stencil inputs (with their 4-cell halo) and of the point inputs into a
// shared-memory stage, and an mbarrier counts the bytes in.  Two stages:
// while shot i is computed, shot i+1's tiles are in flight.  Every field
// carries a zero ghost band and the tensor bounds fill zeros, so no load is
// guarded.  Waits are bounded by a deadline; a timeout sets a device status
// word and the CTA returns.
#include "hv_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace hvk {

using hvi::GH;

namespace {

constexpr float LC1 = (float)(8.0 / 5.0);
constexpr float LC2 = (float)(-1.0 / 5.0);
constexpr float LC3 = (float)(8.0 / 315.0);
constexpr float LC4 = (float)(-1.0 / 560.0);

constexpr int kShotsPerGroup = 8;
constexpr int kTileMenu = 16;      // number of tile configurations (with_cfg)
static_assert(kTileMenu <= kMaxTileMenu, "the bulk-copy descriptors have a slot per configuration");

// BX x BZ threads, each on 4 x RZ points; ST copy stages (shots in flight per
// CTA = ST - 1); GPC shot groups of 8 walked by one CTA.  The last two change
// neither the arithmetic nor its order: every configuration gives bitwise the
// same fields and images.
template <int BX_, int BZ_, int RZ_, int ST_ = 2, int GPC_ = 1>
struct Cfg {
    static constexpr int BX = BX_, BZ = BZ_, RZ = RZ_, ST = ST_, GPC = GPC_;
    static_assert(ST >= 2 && ST <= 4 && GPC >= 1 && GPC <= 4, "pipeline depth and shot groups per CTA");
    static constexpr int NT = BX * BZ;
    static constexpr int TX = 4 * BX, TZ = RZ * BZ;
    static constexpr int W = TX + 2 * GH, H = TZ + 2 * GH;
    static constexpr int W4 = W / 4;
    static constexpr int HALO = W * H * 4;   // bytes of a halo tile (one bulk copy)
    static constexpr int PT = TX * TZ * 4;   // bytes of a point tile
    static constexpr int HALOP = (HALO + 127) / 128 * 128;   // shared-memory slots, 128-byte aligned
    static constexpr int PTP = (PT + 127) / 128 * 128;
};
// The tile menu (the autotuner picks one per kernel kind and problem):
using Cfg64x32 = Cfg<16, 16, 2>;   // 256 threads, 4 x 2 points each
using Cfg32x32 = Cfg<8, 16, 2>;    // 128 threads
using Cfg64x16 = Cfg<16, 8, 2>;    // 128 threads
using Cfg52x26 = Cfg<13, 13, 2>;   // 169 threads; tiles a 104-point padded axis exactly
using Cfg128x16 = Cfg<32, 8, 2>;   // 256 threads
using Cfg64x8 = Cfg<16, 4, 2>;     // 64 threads
using Cfg32x16 = Cfg<8, 8, 2>;     // 64 threads
using Cfg128x8 = Cfg<32, 4, 2>;    // 128 threads
using Cfg32x16s3 = Cfg<8, 8, 2, 3, 1>;     // three stages
using Cfg32x16g4 = Cfg<8, 8, 2, 2, 4>;     // 32 shots per CTA
using Cfg32x16s3g4 = Cfg<8, 8, 2, 3, 4>;
using Cfg128x8s3 = Cfg<32, 4, 2, 3, 1>;
using Cfg128x8g4 = Cfg<32, 4, 2, 2, 4>;
using Cfg128x8s3g4 = Cfg<32, 4, 2, 3, 4>;
using Cfg64x16s3g2 = Cfg<16, 8, 2, 3, 2>;
using Cfg64x8s3g4 = Cfg<16, 4, 2, 3, 4>;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase; false (and the status word set) once wait_ns
// nanoseconds have passed (the handle's wait limit, hv_set_wait_limit).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status, unsigned long long wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > wait_ns) {
            atomicExch(status, HV_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// Programmatic dependent launch.  A step launched with the programmatic
// stream-serialization attribute may start while the previous step's last CTAs
// still run; it reads nothing that an earlier kernel wrote, and writes nothing,
// before grid_dependency_wait() returns (which is when every prerequisite grid
// has completed and its memory operations are visible).  A step lets the next
// one launch once it has passed its own wait, so at most two steps overlap and
// everything before the previous step has finished.  Both are no-ops in a
// kernel launched without the attribute.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Dataflow between steps.  Every CTA adds one to the counter of each (shot
// group, tile) item it finishes, after all its threads' stores (bar.sync, then
// a releasing reduction at GPU scope by thread 0).  A CTA of a later step acquires the
// counters of its tile and the 8 neighbours (the stencil reaches 4 cells,
// less than a tile) until each has reached `need`, the items of all earlier
// steps of the call; the neighbours' earlier steps then are complete too,
// since each of their items waited the same way.  The bulk copies that follow
// read through the async proxy, hence the proxy fence after the acquire.
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void publish_item(int *c)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(c) : "memory");
}

// Thread 0: waits (bounded by wait_ns) until tile `tile` and its neighbours
// have `need` completed items of shot group g.  false after the deadline
// (status set) or when another CTA has already reported an error.
__device__ bool wait_neighbourhood(const int *cnt, int g, int tile, int ntx, int ntiles, int need, int *status,
                                   unsigned long long wait_ns)
{
    const int ntz = ntiles / ntx;
    const int tz = tile / ntx, tx = tile - tz * ntx;
    const int *row = cnt + (size_t)g * ntiles;
    unsigned long long t0 = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dx = -1; dx <= 1; ++dx) {
            const int z = tz + dz, x = tx + dx;
            if (z < 0 || z >= ntz || x < 0 || x >= ntx) continue;
            const int *c = row + z * ntx + x;
            while (ld_acquire(c) < need) {
                if (t0 == 0) t0 = globaltimer();
                if (*(volatile int *)status != 0) return false;
                if (globaltimer() - t0 > wait_ns) {
                    atomicExch(status, HV_ETIMEOUT);
                    return false;
                }
                __nanosleep(128);
            }
        }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// The CTA's wait for the data of earlier steps: tile waits for every shot
// group of shots [s0, s1) in dataflow mode, else the grid-dependency wait.
// false if the CTA must give up (every thread gets the same answer).
__device__ __forceinline__ bool wait_for_inputs(bool flow, const int *cnt, int s0, int s1, int gsz, int tile, int ntx,
                                                int ntiles, int need, int *status, unsigned long long wait_ns)
{
    bool ok = true;
    if (flow) {
        if (threadIdx.x == 0)
            for (int g = s0 / gsz; g * gsz < s1 && ok; ++g)
                ok = wait_neighbourhood(cnt, g, tile, ntx, ntiles, need, status, wait_ns);
    } else {
        grid_dependency_wait();
    }
    return !__syncthreads_or(!ok);
}

// 3D tiled bulk copy global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int z, int f, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(z), "r"(f), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------------ stencil
// The Laplacian sum Lh: the k = 1 term is
// summed over differences from the centre, c1 ((w[+1] - w0) + (w[-1] - w0)),
// the k = 2..4 terms as plain pairs, and the centre coefficient of those terms
// (-4 (c2 + c3 + c4), so that the total centre weight is 4 c0) is added last.
// The k = 1 differences are small and nearly exact for smooth fields; this
// keeps the FP32 wavefield error about 7x below that of the direct sum (the
// same as differencing every term) with 21 instead of 32 operations per point.
constexpr float LCR = (float)(-4.0 * (-1.0 / 5.0 + 8.0 / 315.0 - 1.0 / 560.0));

// ------------------------------------------------------------------ packed FP32
// The stencil arithmetic runs on pairs of neighbouring x points with the
// paired FP32 instructions (add / sub / mul / fma on .f32x2): one instruction
// rounds each lane exactly as its scalar counterpart would, so every lane sees
// the same sequence of correctly rounded operations as a scalar kernel.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b)
{
    unsigned long long x, y, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lo(const float4 &q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi(const float4 &q) { return make_float2(q.z, q.w); }

// Lh at a 4 x RZ block of points of a shared-memory array (4 cells of halo
// around them), as RZ x 2 pairs (points 0, 1 and 2, 3 of each row).  Per lane:
//   d1  = ((w[x-1] - w0) + (w[x+1] - w0)) + ((w[z-1] - w0) + (w[z+1] - w0))
//   acc = c4 ((w[x-4] + w[x+4]) + (w[z-4] + w[z+4]))
//   acc = c3 ((w[x-3] + w[x+3]) + (w[z-3] + w[z+3])) + acc,  then c2 likewise
//   Lh  = c1 d1 + (LCR w0 + acc)
// The z neighbours of a pair are halves of the float4 columns; the x
// neighbours at odd offsets are re-paired from adjacent float4s.  The points
// sit at rows rbase + 4 .. rbase + 3 + RZ and float4 column c4 of an array of
// W4 float4s per row.
template <int RZ>
__device__ __forceinline__ void lap_at(const float *__restrict__ sm, int W4, int rbase, int c4, float2 (&L)[RZ][2],
                                       float2 (&ctr)[RZ][2])
{
    const float4 *s4 = reinterpret_cast<const float4 *>(sm);
    float4 col[RZ + 8];
#pragma unroll
    for (int i = 0; i < RZ + 8; ++i) col[i] = s4[(rbase + i) * W4 + c4];
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int row = rbase + r + GH;
        const float4 xm = s4[row * W4 + c4 - 1];
        const float4 xc = col[r + 4];
        const float4 xp = s4[row * W4 + c4 + 1];
        // e[i] = (v[2i], v[2i+1]), o[i] = (v[2i+1], v[2i+2]) over v = xm | xc | xp
        const float2 e[6] = {lo(xm), hi(xm), lo(xc), hi(xc), lo(xp), hi(xp)};
        const float2 o[5] = {make_float2(xm.y, xm.z), make_float2(xm.w, xc.x), make_float2(xc.y, xc.z),
                             make_float2(xc.w, xp.x), make_float2(xp.y, xp.z)};
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            // x neighbour at offset k - 4 of lanes 2pr, 2pr+1; z neighbour in column i
            auto hx = [&](int k) { return (k & 1) ? o[(k - 1) / 2 + pr] : e[k / 2 + pr]; };
            auto zc = [&](int i) { return pr == 0 ? lo(col[i]) : hi(col[i]); };
            const float2 cz = zc(r + 4);
            const float2 d1 = f2add(f2add(f2sub(hx(3), cz), f2sub(hx(5), cz)),
                                    f2add(f2sub(zc(r + 3), cz), f2sub(zc(r + 5), cz)));
            float2 acc = f2mul(splat(LC4), f2add(f2add(hx(0), hx(8)), f2add(zc(r), zc(r + 8))));
            acc = f2fma(splat(LC3), f2add(f2add(hx(1), hx(7)), f2add(zc(r + 1), zc(r + 7))), acc);
            acc = f2fma(splat(LC2), f2add(f2add(hx(2), hx(6)), f2add(zc(r + 2), zc(r + 6))), acc);
            acc = f2fma(splat(LCR), cz, acc);
            L[r][pr] = f2fma(splat(LC1), d1, acc);
            ctr[r][pr] = cz;
        }
    }
}

// The thread's block of a CTA tile: rows tz*RZ .. of a [H][W] halo tile, float4 column tx + 1.
template <class C>
__device__ __forceinline__ void lap_block(const float *__restrict__ sm, int tx, int tz, float2 (&L)[C::RZ][2],
                                          float2 (&ctr)[C::RZ][2])
{
    lap_at<C::RZ>(sm, C::W4, tz * C::RZ, tx + 1, L, ctr);
}

// Sponge factors of one row of the thread's block, as pairs: inv = 1 / (1 + a)
// and nom = a - 1 (= -(1 - a) exactly) with a = max(a_z, a_x).
__device__ __forceinline__ void sponge_row(const float *az, int z, int NZ, const float (&axv)[4], float2 (&inv)[2],
                                           float2 (&nom)[2])
{
    const float azv = az[min(z, NZ - 1)];
    float iv[4], nm[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float a = fmaxf(azv, axv[c]);
        iv[c] = __frcp_rn(1.0f + a);
        nm[c] = a - 1.0f;
    }
    inv[0] = make_float2(iv[0], iv[1]);
    inv[1] = make_float2(iv[2], iv[3]);
    nom[0] = make_float2(nm[0], nm[1]);
    nom[1] = make_float2(nm[2], nm[3]);
}

// The same factors from values fixed per thread: the damping rates of the
// thread's RZ rows and 4 columns and their reciprocal factors 1 / (1 + a),
// computed once per CTA.  Rounding is monotone, so 1 / (1 + max(az, ax))
// rounded equals min(1 / (1 + az), 1 / (1 + ax)) rounded: bitwise the values
// sponge_row computes, without a load or a division per shot.
template <int RZ>
struct SpongeRegs {
    float az[RZ], iz[RZ], ax[4], ix[4];
};

template <int RZ>
__device__ __forceinline__ void sponge_regs(SpongeRegs<RZ> &sp, const float *az, const float *ax, int zrow0, int xb,
                                            int NZ, int NX)
{
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        sp.az[r] = az[min(zrow0 + r, NZ - 1)];
        sp.iz[r] = __frcp_rn(1.0f + sp.az[r]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        sp.ax[c] = ax[min(xb + c, NX - 1)];
        sp.ix[c] = __frcp_rn(1.0f + sp.ax[c]);
    }
}

template <int RZ>
__device__ __forceinline__ void sponge_row(const SpongeRegs<RZ> &sp, int r, float2 (&inv)[2], float2 (&nom)[2])
{
    float iv[4], nm[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        iv[c] = fminf(sp.iz[r], sp.ix[c]);
        nm[c] = fmaxf(sp.az[r], sp.ax[c]) - 1.0f;
    }
    inv[0] = make_float2(iv[0], iv[1]);
    inv[1] = make_float2(iv[2], iv[3]);
    nom[0] = make_float2(nm[0], nm[1]);
    nom[1] = make_float2(nm[2], nm[3]);
}

__device__ __forceinline__ void f4(const float *p, float2 (&o)[2])
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = lo(v);
    o[1] = hi(v);
}

// Store 4 consecutive x values at padded column x.. (skipping x >= NX).
__device__ __forceinline__ void st4(float *p, const float2 (&o)[2], int x, int NX)
{
    if (x + 3 < NX) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    } else {
        const float w[4] = {o[0].x, o[0].y, o[1].x, o[1].y};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (x + c < NX) p[c] = w[c];
    }
}

struct Geo {
    int P, NZ, NX, nz, nx, nb, ntx, ntiles;
    unsigned long long fsize;   // floats per field
};

struct FwdParams {
    CUtensorMap map_halo;       // box (TX+8) x (TZ+8) x 1
    CUtensorMap map_pt;         // box TX x TZ x 1
    float *ws;                  // workspace base (field 0)
    int f_ucur, f_uprev, f_unext;   // field-batch starts (f_unext < 0: do not write u)
    const int *slot_join;       // per-model step counters (no Born fields), or nullptr (see k_fwd)
    int f_C, f_b, f_du, f_dio;      // coefficient fields and Born field batches
    float *d_u, *d_du;
    const float *az, *ax, *wavelet;
    const int *src_zx, *rt_off, *rt_rec, *rt_pos;
    int *status;
    unsigned long long wait_ns;  // limit of every device wait [ns]
    int n, nt, nr, ns, k, spg, gsz;
    int *cnt;                   // step counters per (shot group, tile), or nullptr
    int need, flow;             // dataflow ordering (StepDeps)
    Geo g;
};

constexpr int kMaxSpg = 32;   // shots per CTA, upper bound (per-CTA shot tables)

// Per-CTA copy of the shot tables of its shots: source node and the range of
// this tile's receivers, for every shot (read once instead of once per shot).
struct ShotTables {
    int sz[kMaxSpg], sx[kMaxSpg], rb[kMaxSpg], re[kMaxSpg];
};
constexpr int kTablesBytes = 512;
static_assert(sizeof(ShotTables) <= kTablesBytes, "shot tables fit their shared-memory slot");
static_assert(4 * kShotsPerGroup <= kMaxSpg, "four shot groups fit the shot tables");

// Shared memory: ST stages, the coefficient tiles, ST + 1 mbarriers, the shot tables.
template <class C, bool BORN>
struct FwdSmem {
    static constexpr int STAGE = C::HALOP + C::PTP + (BORN ? C::HALOP + C::PTP : 0);
    static constexpr int STAGE_TX = C::HALO + C::PT + (BORN ? C::HALO + C::PT : 0);   // bytes each stage receives
    static constexpr int COEF = C::PTP * (BORN ? 2 : 1);
    static constexpr int COEF_TX = C::PT * (BORN ? 2 : 1);
    static constexpr int BARS = C::ST * STAGE + COEF;
    static constexpr int BYTES = BARS + 64 + kTablesBytes;
};

__device__ __forceinline__ void load_shot_tables(ShotTables &t, const int *src_zx, const int *rt_off, int s0, int n,
                                                 int tile, int ntiles)
{
    const int i = threadIdx.x;
    if (i < n) {
        const int s = s0 + i;
        t.sz[i] = src_zx[2 * s];
        t.sx[i] = src_zx[2 * s + 1];
        t.rb[i] = rt_off[s * (ntiles + 1) + tile];
        t.re[i] = rt_off[s * (ntiles + 1) + tile + 1];
    }
}

// Adds s_n to Q at the source node if it lies in the thread's block.
template <class C>
__device__ __forceinline__ void add_source(float2 (&Q)[C::RZ][2], int zrow0, int xb, int sz, int sx, float wav)
{
    const int dz = sz - zrow0, dx = sx - xb;
    if ((unsigned)dz < (unsigned)C::RZ && (unsigned)dx < 4u) {
#pragma unroll
        for (int r = 0; r < C::RZ; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (r == dz && c == dx) {
                    if (c & 1) Q[r][c >> 1].y += wav;
                    else Q[r][c >> 1].x += wav;
                }
    }
}

// o = (2 w - (1 - a) w_prev + C q) / (1 + a); a = 0 (SP false) off the sponge,
// where 2 w - w_prev is one rounding (2 w is exact).  Every operation is an
// explicit correctly rounded one: the compiler has no contraction freedom, so
// each tile shape computes bitwise the same values.
template <bool SP>
__device__ __forceinline__ float2 leapfrog(float2 w, float2 wprev, float2 cc, float2 q, float2 inv, float2 nom)
{
    if constexpr (SP) return f2mul(inv, f2fma(cc, q, f2fma(nom, wprev, f2add(w, w))));
    else return f2fma(cc, q, f2sub(f2add(w, w), wprev));
}

// After a failed wait: wait (bounded) for the copies of items [from, to) still
// in flight, so that none lands after the CTA has exited.
template <int ST>
__device__ __forceinline__ void drain_stages(uint64_t *bars, int from, int to, int *status, unsigned long long wait_ns)
{
    for (int q = from; q < to; ++q) mbar_wait(&bars[q % ST], (q / ST) & 1, status, wait_ns);
}

// One forward time step.  grid = (ntiles, k, shot groups).  With Born fields
// y is the vector j (vector 0 writes u^{n+1}; every CTA recomputes
// Q^n = Lh u^n + s_n from its own tile); without them y selects one of k
// models, each with its own coefficient field, field batch [ns] and data
// (several models in one sweep, hv_misfit_models).  With slot_join (no Born
// fields) every model has its own step counter: p.n counts the launches, model
// j takes its step p.n - slot_join[j] (none if that is outside [0, nt), e.g. a
// free slot, slot_join 1 << 30 > p.n) and its three time levels rotate through a
// ring of three field batches of its own starting 3 ns j fields after f_ucur.
template <class C, bool BORN>
__global__ void __launch_bounds__(C::NT, 2) k_fwd(const __grid_constant__ FwdParams p)
{
    using S = FwdSmem<C, BORN>;
    extern __shared__ __align__(128) unsigned char smem[];
    float *sC = reinterpret_cast<float *>(smem + C::ST * S::STAGE);
    float *sB = sC + C::PTP / 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BARS);   // [0, ST): stages, [ST]: coefficients
    ShotTables &tab = *reinterpret_cast<ShotTables *>(smem + S::BARS + 64);

    const int tile = blockIdx.x, j = blockIdx.y, grp = blockIdx.z;
    const int tzi = tile / p.g.ntx, txi = tile - tzi * p.g.ntx;
    const int z0 = tzi * C::TZ, x0 = txi * C::TX;
    const int s0 = grp * p.spg, s1 = min(p.ns, s0 + p.spg), nitems = s1 - s0;
    const int tx = threadIdx.x % C::BX, tz = threadIdx.x / C::BX;
    const int xb = x0 + 4 * tx, zrow0 = z0 + tz * C::RZ;
    const int mo = BORN ? 0 : j;                    // the model
    int n = p.n, fcur = p.f_ucur + mo * p.ns, fprev = p.f_uprev + mo * p.ns, fnext = p.f_unext + mo * p.ns;
    if constexpr (!BORN) {
        if (p.slot_join) {                          // read before the grid-dependency wait: written by an earlier copy
            n = p.n - p.slot_join[j];
            if (n < 0 || n >= p.nt) return;         // the slot takes no step in this launch
            const int ring = p.f_ucur + 3 * p.ns * j;
            fcur = ring + (n % 3) * p.ns;
            fprev = ring + ((n + 2) % 3) * p.ns;
            fnext = ring + ((n + 1) % 3) * p.ns;
        }
    }
    const bool write_u = p.f_unext >= 0 && (!BORN || j == 0);

    auto issue = [&](int i) {
        const int st = i % C::ST, s = s0 + i;
        unsigned char *base = smem + st * S::STAGE;
        mbar_expect_tx(&bars[st], S::STAGE_TX);
        tma_load(base, &p.map_halo, x0, z0, fcur + s, &bars[st]);
        tma_load(base + C::HALOP, &p.map_pt, x0 + GH, z0 + GH, fprev + s, &bars[st]);
        if constexpr (BORN) {
            const int fo = j * p.ns + s;
            tma_load(base + C::HALOP + C::PTP, &p.map_halo, x0, z0, p.f_du + fo, &bars[st]);
            tma_load(base + 2 * C::HALOP + C::PTP, &p.map_pt, x0 + GH, z0 + GH, p.f_dio + fo, &bars[st]);
        }
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q <= C::ST; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    // From here on the fields of earlier steps are complete and visible.
    if (!wait_for_inputs(p.flow, p.cnt, s0, s1, p.gsz, tile, p.g.ntx, p.g.ntiles, p.need, p.status, p.wait_ns)) return;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bars[C::ST], S::COEF_TX);
        tma_load(sC, &p.map_pt, x0 + GH, z0 + GH, p.f_C + mo, &bars[C::ST]);
        if constexpr (BORN) tma_load(sB, &p.map_pt, x0 + GH, z0 + GH, p.f_b + j, &bars[C::ST]);
        for (int q = 0; q < C::ST && q < nitems; ++q) issue(q);
    }
    allow_dependent_launch();
    // Set-up from the handle's constant tables (written before any step) while
    // the first copies are in flight; the barrier after the coefficient wait
    // publishes the shot tables.
    load_shot_tables(tab, p.src_zx, p.rt_off, s0, nitems, tile, p.g.ntiles);
    // Tiles entirely inside the interior have a = 0 and take the short update.
    const bool sponge = !(z0 >= p.g.nb && z0 + C::TZ <= p.g.nb + p.g.nz && x0 >= p.g.nb &&
                          x0 + C::TX <= p.g.nb + p.g.nx);
    SpongeRegs<C::RZ> spr{};
    if (sponge) sponge_regs<C::RZ>(spr, p.az, p.ax, zrow0, xb, p.g.NZ, p.g.NX);
    const float wav = p.wavelet[n];

    bool ok = mbar_wait(&bars[C::ST], 0, p.status, p.wait_ns);
    if (__syncthreads_or(!ok)) {
        drain_stages<C::ST>(bars, 0, min(C::ST, nitems), p.status, p.wait_ns);
        return;
    }

    auto run = [&](auto sp_tag) {
        constexpr bool SP = decltype(sp_tag)::value;
        for (int i = 0; i < nitems; ++i) {
            const int st = i % C::ST, s = s0 + i;
            ok = mbar_wait(&bars[st], (i / C::ST) & 1, p.status, p.wait_ns);
            if (__syncthreads_or(!ok)) {
                // a copy did not arrive: let the other stages drain (bounded), then give up
                drain_stages<C::ST>(bars, i + 1, min(i + C::ST, nitems), p.status, p.wait_ns);
                return;
            }
            const unsigned char *base = smem + st * S::STAGE;
            const float *sU = reinterpret_cast<const float *>(base);
            const float *sUp = reinterpret_cast<const float *>(base + C::HALOP);

            float2 Q[C::RZ][2], uc[C::RZ][2];
            lap_block<C>(sU, tx, tz, Q, uc);
            add_source<C>(Q, zrow0, xb, tab.sz[i], tab.sx[i], wav);
            const int rb = tab.rb[i], re = tab.re[i];
            if (write_u) {
                float *un = p.ws + (unsigned long long)(fnext + s) * p.g.fsize;
#pragma unroll
                for (int r = 0; r < C::RZ; ++r) {
                    const int z = zrow0 + r;
                    float2 up[2], cc[2], inv[2] = {}, nom[2] = {}, o[2];
                    f4(sUp + (tz * C::RZ + r) * C::TX + 4 * tx, up);
                    f4(sC + (tz * C::RZ + r) * C::TX + 4 * tx, cc);
                    if constexpr (SP) sponge_row<C::RZ>(spr, r, inv, nom);
#pragma unroll
                    for (int h = 0; h < 2; ++h) o[h] = leapfrog<SP>(uc[r][h], up[h], cc[h], Q[r][h], inv[h], nom[h]);
                    if (z < p.g.NZ && xb < p.g.NX) st4(un + (size_t)(z + GH) * p.g.P + (xb + GH), o, xb, p.g.NX);
                }
                if (p.d_u && rb < re) {
                    __syncthreads();
                    for (int q = rb + threadIdx.x; q < re; q += C::NT)
                        p.d_u[((size_t)(mo * p.ns + s) * p.nt + n) * p.nr + p.rt_rec[s * p.nr + q]] = un[p.rt_pos[s * p.nr + q]];
                }
            }
            if constexpr (BORN) {
                const float *sD = reinterpret_cast<const float *>(base + C::HALOP + C::PTP);
                const float *sDp = reinterpret_cast<const float *>(base + 2 * C::HALOP + C::PTP);
                float2 Ld[C::RZ][2], dc[C::RZ][2];
                lap_block<C>(sD, tx, tz, Ld, dc);
                const int fo = j * p.ns + s;
                float *dn = p.ws + (unsigned long long)(p.f_dio + fo) * p.g.fsize;
#pragma unroll
                for (int r = 0; r < C::RZ; ++r) {
                    const int z = zrow0 + r;
                    float2 dp[2], cc[2], bb[2], inv[2] = {}, nom[2] = {}, o[2];
                    f4(sDp + (tz * C::RZ + r) * C::TX + 4 * tx, dp);
                    f4(sC + (tz * C::RZ + r) * C::TX + 4 * tx, cc);
                    f4(sB + (tz * C::RZ + r) * C::TX + 4 * tx, bb);
                    if constexpr (SP) sponge_row<C::RZ>(spr, r, inv, nom);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        o[h] = leapfrog<SP>(dc[r][h], dp[h], cc[h], f2fma(bb[h], Q[r][h], Ld[r][h]), inv[h], nom[h]);
                    if (z < p.g.NZ && xb < p.g.NX) st4(dn + (size_t)(z + GH) * p.g.P + (xb + GH), o, xb, p.g.NX);
                }
                if (p.d_du && rb < re) {
                    __syncthreads();
                    for (int q = rb + threadIdx.x; q < re; q += C::NT)
                        p.d_du[((size_t)fo * p.nt + p.n) * p.nr + p.rt_rec[s * p.nr + q]] = dn[p.rt_pos[s * p.nr + q]];
                }
            }
            __syncthreads();                       // every thread is done with stage st
            if (threadIdx.x == 0) {
                if (p.cnt && ((s + 1) % p.gsz == 0 || i + 1 == nitems))
                    publish_item(p.cnt + (size_t)(s / p.gsz) * p.g.ntiles + tile);
                if (i + C::ST < nitems) issue(i + C::ST);
            }
        }
    };
    if (sponge) run(std::true_type{});
    else run(std::false_type{});
}

// ------------------------------------------------------------------ two fused steps
// Two forward steps (no Born field, no receivers: the recomputation of the
// reversal) in one pass over the fields.  The CTA computes u^{n+1} on its tile
// extended by the 4-cell stencil reach (region E), from u^n with an 8-cell halo
// and u^{n-1} on E; the extended ring is recomputed with exactly the arithmetic
// of the single step (and set to zero off the padded grid, as the ghost band
// is), so u^{n+1} and u^{n+2} are bitwise those of two single steps.  Reads
// u^n and u^{n-1} once and writes u^{n+1} and u^{n+2}: 16 bytes per point for
// two steps instead of 24 (plus the coefficient field, shared by the shots).
struct Fwd2Params {
    CUtensorMap map_halo;       // box (TX+8) x (TZ+8): u^{n-1} and C on E
    CUtensorMap map_halo8;      // box (TX+16) x (TZ+16): u^n
    float *ws;
    int f_ucur, f_uprev, f_unext1, f_unext2, f_C;
    const float *az, *ax, *wavelet;
    const int *src_zx, *rt_off;
    int *status;
    unsigned long long wait_ns;
    int n, ns, spg;
    Geo g;
};

template <class C>
struct Fwd2Smem {
    static constexpr int W8 = C::TX + 16, H8 = C::TZ + 16;
    static constexpr int H8B = W8 * H8 * 4, H8P = (H8B + 127) / 128 * 128;
    static constexpr int STAGE = H8P + C::HALOP;           // u^n (halo 8), u^{n-1} on E
    static constexpr int STAGE_TX = H8B + C::HALO;
    static constexpr int BARS = C::ST * STAGE + 2 * C::HALOP;   // + C on E, u^{n+1} on E
    static constexpr int BYTES = BARS + 64 + kTablesBytes;
};

template <class C>
__global__ void __launch_bounds__(C::NT, 1) k_fwd2(const __grid_constant__ Fwd2Params p)
{
    using S = Fwd2Smem<C>;
    constexpr int EBX = C::BX + 2, EBZ = (C::TZ + 8) / C::RZ, NEB = EBX * EBZ;   // 4 x RZ blocks of E
    static_assert((C::TZ + 8) % C::RZ == 0, "E rows split into whole register blocks");
    extern __shared__ __align__(128) unsigned char smem[];
    float *sCe = reinterpret_cast<float *>(smem + C::ST * S::STAGE);   // C on E, [H][W]
    float *sU1 = sCe + C::HALOP / 4;                                   // u^{n+1} on E, [H][W]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BARS);
    ShotTables &tab = *reinterpret_cast<ShotTables *>(smem + S::BARS + 64);

    const int tile = blockIdx.x, grp = blockIdx.z;
    const int tzi = tile / p.g.ntx, txi = tile - tzi * p.g.ntx;
    const int z0 = tzi * C::TZ, x0 = txi * C::TX;
    const int s0 = grp * p.spg, s1 = min(p.ns, s0 + p.spg), nitems = s1 - s0;
    const int tx = threadIdx.x % C::BX, tz = threadIdx.x / C::BX;
    const int xb = x0 + 4 * tx, zrow0 = z0 + tz * C::RZ;

    auto issue = [&](int i) {
        const int st = i % C::ST, s = s0 + i;
        unsigned char *base = smem + st * S::STAGE;
        mbar_expect_tx(&bars[st], S::STAGE_TX);
        tma_load(base, &p.map_halo8, x0 - GH, z0 - GH, p.f_ucur + s, &bars[st]);
        tma_load(base + S::H8P, &p.map_halo, x0, z0, p.f_uprev + s, &bars[st]);
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q <= C::ST; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    load_shot_tables(tab, p.src_zx, p.rt_off, s0, nitems, tile, p.g.ntiles);
    // Sponge flags: E (tile + 4) for the first step, the tile for the second.
    const bool sponge1 = !(z0 - GH >= p.g.nb && z0 + C::TZ + GH <= p.g.nb + p.g.nz && x0 - GH >= p.g.nb &&
                           x0 + C::TX + GH <= p.g.nb + p.g.nx);
    const bool sponge2 = !(z0 >= p.g.nb && z0 + C::TZ <= p.g.nb + p.g.nz && x0 >= p.g.nb &&
                           x0 + C::TX <= p.g.nb + p.g.nx);
    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    if (sponge2)
#pragma unroll
        for (int c = 0; c < 4; ++c) axv[c] = p.ax[min(xb + c, p.g.NX - 1)];
    const float wav1 = p.wavelet[p.n], wav2 = p.wavelet[p.n + 1];
    grid_dependency_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bars[C::ST], C::HALO);
        tma_load(sCe, &p.map_halo, x0, z0, p.f_C, &bars[C::ST]);
        for (int q = 0; q < C::ST && q < nitems; ++q) issue(q);
    }
    allow_dependent_launch();

    bool ok = mbar_wait(&bars[C::ST], 0, p.status, p.wait_ns);
    if (__syncthreads_or(!ok)) {
        drain_stages<C::ST>(bars, 0, min(C::ST, nitems), p.status, p.wait_ns);
        return;
    }

    auto run = [&](auto sp1_tag, auto sp2_tag) {
        constexpr bool SP1 = decltype(sp1_tag)::value, SP2 = decltype(sp2_tag)::value;
        for (int i = 0; i < nitems; ++i) {
            const int st = i % C::ST, s = s0 + i;
            ok = mbar_wait(&bars[st], (i / C::ST) & 1, p.status, p.wait_ns);
            if (__syncthreads_or(!ok)) {
                drain_stages<C::ST>(bars, i + 1, min(i + C::ST, nitems), p.status, p.wait_ns);
                return;
            }
            const unsigned char *base = smem + st * S::STAGE;
            const float *sU8 = reinterpret_cast<const float *>(base);
            const float *sUp = reinterpret_cast<const float *>(base + S::H8P);
            float *u1g = p.ws + (unsigned long long)(p.f_unext1 + s) * p.g.fsize;
            // ---- step n -> n+1 on E
            for (int eb = threadIdx.x; eb < NEB; eb += C::NT) {
                const int ebx = eb % EBX, ebz = eb / EBX;
                const int ez0 = ebz * C::RZ, ex0 = 4 * ebx;            // E coordinates of the block
                const int pz0 = z0 - GH + ez0, px0 = x0 - GH + ex0;    // padded-grid coordinates
                float2 Q[C::RZ][2], uc[C::RZ][2];
                lap_at<C::RZ>(sU8, S::W8 / 4, ez0, ebx + 1, Q, uc);
                add_source<C>(Q, pz0, px0, tab.sz[i], tab.sx[i], wav1);
                float axe[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) axe[c] = SP1 ? p.ax[min(max(px0 + c, 0), p.g.NX - 1)] : 0.0f;
#pragma unroll
                for (int r = 0; r < C::RZ; ++r) {
                    const int pz = pz0 + r, er = ez0 + r;
                    float2 up[2], cc[2], inv[2] = {}, nom[2] = {}, o[2];
                    f4(sUp + er * C::W + ex0, up);
                    f4(sCe + er * C::W + ex0, cc);
                    if constexpr (SP1) sponge_row(p.az, min(max(pz, 0), p.g.NZ - 1), p.g.NZ, axe, inv, nom);
#pragma unroll
                    for (int h = 0; h < 2; ++h) o[h] = leapfrog<SP1>(uc[r][h], up[h], cc[h], Q[r][h], inv[h], nom[h]);
                    float w[4] = {o[0].x, o[0].y, o[1].x, o[1].y};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (pz < 0 || pz >= p.g.NZ || px0 + c < 0 || px0 + c >= p.g.NX) w[c] = 0.0f;   // ghost band
                    *reinterpret_cast<float4 *>(sU1 + er * C::W + ex0) = make_float4(w[0], w[1], w[2], w[3]);
                    if (er >= GH && er < C::TZ + GH && ebx >= 1 && ebx <= C::BX && pz < p.g.NZ && px0 < p.g.NX) {
                        const float2 wo[2] = {make_float2(w[0], w[1]), make_float2(w[2], w[3])};
                        st4(u1g + (size_t)(pz + GH) * p.g.P + (px0 + GH), wo, px0, p.g.NX);
                    }
                }
            }
            __syncthreads();
            // ---- step n+1 -> n+2 on the tile
            {
                float2 Q[C::RZ][2], uc[C::RZ][2];
                lap_block<C>(sU1, tx, tz, Q, uc);
                add_source<C>(Q, zrow0, xb, tab.sz[i], tab.sx[i], wav2);
                float *u2g = p.ws + (unsigned long long)(p.f_unext2 + s) * p.g.fsize;
#pragma unroll
                for (int r = 0; r < C::RZ; ++r) {
                    const int z = zrow0 + r;
                    float2 up[2], cc[2], inv[2] = {}, nom[2] = {}, o[2];
                    f4(sU8 + (tz * C::RZ + r + 2 * GH) * S::W8 + 4 * tx + 2 * GH, up);
                    f4(sCe + (tz * C::RZ + r + GH) * C::W + 4 * tx + GH, cc);
                    if constexpr (SP2) sponge_row(p.az, z, p.g.NZ, axv, inv, nom);
#pragma unroll
                    for (int h = 0; h < 2; ++h) o[h] = leapfrog<SP2>(uc[r][h], up[h], cc[h], Q[r][h], inv[h], nom[h]);
                    if (z < p.g.NZ && xb < p.g.NX) st4(u2g + (size_t)(z + GH) * p.g.P + (xb + GH), o, xb, p.g.NX);
                }
            }
            __syncthreads();                       // stage st and sU1 are free again
            if (threadIdx.x == 0 && i + C::ST < nitems) issue(i + C::ST);
        }
    };
    if (sponge2) run(std::true_type{}, std::true_type{});
    else if (sponge1) run(std::true_type{}, std::false_type{});
    else run(std::false_type{}, std::false_type{});
}

struct AdjParams {
    CUtensorMap map_halo, map_pt;
    float *ws;
    int f_u, f_lam1, f_lamio, f_C;
    const float *r;
    unsigned long long r_vstride;
    float rscale;
    double *img;    // [G][k][fsize] double-float (hi, lo) pairs, 8 bytes per point
    const float *az, *ax, *wavelet;
    const int *src_zx, *rt_off, *rt_rec, *rt_pos;
    int *status;
    unsigned long long wait_ns;
    int n, nt, nr, ns, k, spg, gsz;
    int *cnt;
    int need, flow;
    Geo g;
};

template <class C>
struct AdjSmem {
    static constexpr int STAGE = 2 * C::HALOP + C::PTP;
    static constexpr int STAGE_TX = 2 * C::HALO + C::PT;
    static constexpr int BARS = C::ST * STAGE + C::PTP /* C */ + C::PTP /* sources */;
    static constexpr int BYTES = BARS + 64 + kTablesBytes;
};

// One adjoint time step with zero-lag imaging.  grid = (ntiles, k, blocks of
// GPC shot groups); for each group of 8 shots the CTA sums the shots' image
// contributions in shot order and adds them to the group's double-float partial image
// once per step.  IMG64 (the precision check of hv_set_image_precision): each
// shot's product lam^n Q^n, exact in FP64, is added to the group's FP64 image
// instead (the CTA owns its tile's points of that image).
template <class C, bool IMG64 = false>
__global__ void __launch_bounds__(C::NT, C::NT <= 64 ? 8 : C::NT <= 128 ? 4 : 2) k_adj(const __grid_constant__ AdjParams p)
{
    using S = AdjSmem<C>;
    extern __shared__ __align__(128) unsigned char smem[];
    float *sC = reinterpret_cast<float *>(smem + C::ST * S::STAGE);
    float *ssrc = sC + C::PTP / 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::BARS);   // [0, ST): stages, [ST]: C
    ShotTables &tab = *reinterpret_cast<ShotTables *>(smem + S::BARS + 64);

    const int tile = blockIdx.x, j = blockIdx.y, grp = blockIdx.z;
    const int tzi = tile / p.g.ntx, txi = tile - tzi * p.g.ntx;
    const int z0 = tzi * C::TZ, x0 = txi * C::TX;
    const int s0 = grp * p.spg, s1 = min(p.ns, s0 + p.spg), nitems = s1 - s0;
    const int tx = threadIdx.x % C::BX, tz = threadIdx.x / C::BX;
    const int xb = x0 + 4 * tx, zrow0 = z0 + tz * C::RZ;

    auto issue = [&](int i) {
        const int st = i % C::ST, s = s0 + i;
        unsigned char *base = smem + st * S::STAGE;
        const int fo = j * p.ns + s;
        mbar_expect_tx(&bars[st], S::STAGE_TX);
        tma_load(base, &p.map_halo, x0, z0, p.f_u + s, &bars[st]);
        tma_load(base + C::HALOP, &p.map_halo, x0, z0, p.f_lam1 + fo, &bars[st]);
        tma_load(base + 2 * C::HALOP, &p.map_pt, x0 + GH, z0 + GH, p.f_lamio + fo, &bars[st]);
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q <= C::ST; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    if (!wait_for_inputs(p.flow, p.cnt, s0, s1, p.gsz, tile, p.g.ntx, p.g.ntiles, p.need, p.status, p.wait_ns)) return;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bars[C::ST], C::PT);
        tma_load(sC, &p.map_pt, x0 + GH, z0 + GH, p.f_C, &bars[C::ST]);
        for (int q = 0; q < C::ST && q < nitems; ++q) issue(q);
    }
    allow_dependent_launch();
    // constant tables while the first copies are in flight (published by the barrier after the C wait)
    load_shot_tables(tab, p.src_zx, p.rt_off, s0, nitems, tile, p.g.ntiles);
    const bool sponge = !(z0 >= p.g.nb && z0 + C::TZ <= p.g.nb + p.g.nz && x0 >= p.g.nb &&
                          x0 + C::TX <= p.g.nb + p.g.nx);
    SpongeRegs<C::RZ> spr{};
    if (sponge) sponge_regs<C::RZ>(spr, p.az, p.ax, zrow0, xb, p.g.NZ, p.g.NX);
    const float wav = p.wavelet[p.n];
    // This step's image contribution of the CTA's shots, summed in shot order
    // in FP32 (at most 8 terms); it is added to the double-float image once per step.
    // Double-precision arithmetic is slow on this part, so none runs per shot.
    float2 acc[C::RZ][2];
#pragma unroll
    for (int r = 0; r < C::RZ; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) acc[r][h] = make_float2(0.0f, 0.0f);

    // Adds the FP32 partial of a finished group of shots to that group's image.
    // The image is held as double-float pairs (hi, lo) and added to by TwoSum on
    // the FP32 pipe -- about 2^-44 relative accuracy, where FP64 arithmetic (and
    // its conversions) would run on this part's slow FP64 pipe; k_fold_g sums
    // the pairs in FP64.
    auto add_df = [](float2 &v, float a) {
        const float s = __fadd_rn(v.x, a), bv = __fsub_rn(s, v.x);
        v.y = __fadd_rn(v.y, __fadd_rn(__fsub_rn(v.x, __fsub_rn(s, bv)), __fsub_rn(a, bv)));
        v.x = s;
    };
    // The group's image words under the thread's full-width rows are loaded when
    // the group's first shot starts, so that the flush does not wait on them.
    float4 imv[C::RZ][2];
    auto img_of = [&](int group) {
        return reinterpret_cast<float2 *>(p.img) + ((size_t)group * p.k + j) * p.g.fsize;
    };
    auto prefetch = [&](int group) {
        const float2 *im = img_of(group);
#pragma unroll
        for (int r = 0; r < C::RZ; ++r) {
            const int z = zrow0 + r;
            if (z < p.g.NZ && xb + 3 < p.g.NX) {
                const float4 *q4 = reinterpret_cast<const float4 *>(im + (size_t)(z + GH) * p.g.P + (xb + GH));
                imv[r][0] = q4[0];
                imv[r][1] = q4[1];
            }
        }
    };
    auto flush = [&](int group) {
        float2 *im = img_of(group);
#pragma unroll
        for (int r = 0; r < C::RZ; ++r) {
            const int z = zrow0 + r;
            if (z < p.g.NZ && xb < p.g.NX) {
                const size_t off = (size_t)(z + GH) * p.g.P + (xb + GH);   // a multiple of 4 pairs: 32-byte aligned
                const float a4[4] = {acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y};
                if (xb + 3 < p.g.NX) {
                    float4 *q4 = reinterpret_cast<float4 *>(im + off);
                    const float4 w0 = imv[r][0], w1 = imv[r][1];
                    float2 v[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                                   make_float2(w1.z, w1.w)};
#pragma unroll
                    for (int c = 0; c < 4; ++c) add_df(v[c], a4[c]);
                    q4[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
                    q4[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (xb + c < p.g.NX) {
                            float2 v = im[off + c];
                            add_df(v, a4[c]);
                            im[off + c] = v;
                        }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) acc[r][h] = make_float2(0.0f, 0.0f);
        }
    };

    if (!IMG64 && nitems > 0) prefetch(s0 / p.gsz);
    bool ok = mbar_wait(&bars[C::ST], 0, p.status, p.wait_ns);
    if (__syncthreads_or(!ok)) {
        drain_stages<C::ST>(bars, 0, min(C::ST, nitems), p.status, p.wait_ns);
        return;
    }

    auto run = [&](auto sp_tag) -> bool {
        constexpr bool SP = decltype(sp_tag)::value;
        for (int i = 0; i < nitems; ++i) {
            const int st = i % C::ST, s = s0 + i;
            const int fo = j * p.ns + s;
            const int rb = tab.rb[i], re = tab.re[i];
            if (!IMG64 && i > 0 && s % p.gsz == 0) prefetch(s / p.gsz);
            if (rb < re) {                         // receivers in this tile: stage their sources
                for (int q = threadIdx.x; q < C::TZ * C::TX; q += C::NT) ssrc[q] = 0.0f;
                __syncthreads();
                const float *rs = p.r + (size_t)j * p.r_vstride + ((size_t)s * p.nt + p.n) * p.nr;
                for (int q = rb + threadIdx.x; q < re; q += C::NT) {
                    const int pos = p.rt_pos[s * p.nr + q];
                    const int zz = pos / p.g.P - GH - z0, xx = pos % p.g.P - GH - x0;
                    ssrc[zz * C::TX + xx] = p.rscale * rs[p.rt_rec[s * p.nr + q]];
                }
            }
            ok = mbar_wait(&bars[st], (i / C::ST) & 1, p.status, p.wait_ns);
            if (__syncthreads_or(!ok)) {
                drain_stages<C::ST>(bars, i + 1, min(i + C::ST, nitems), p.status, p.wait_ns);
                return false;
            }
            const unsigned char *base = smem + st * S::STAGE;
            const float *sU = reinterpret_cast<const float *>(base);
            const float *sL1 = reinterpret_cast<const float *>(base + C::HALOP);
            const float *sL2 = reinterpret_cast<const float *>(base + 2 * C::HALOP);
            float2 Qu[C::RZ][2], ucen[C::RZ][2], Ll[C::RZ][2], lc[C::RZ][2];
            lap_block<C>(sU, tx, tz, Qu, ucen);
            add_source<C>(Qu, zrow0, xb, tab.sz[i], tab.sx[i], wav);
            lap_block<C>(sL1, tx, tz, Ll, lc);
            float *ln = p.ws + (unsigned long long)(p.f_lamio + fo) * p.g.fsize;
#pragma unroll
            for (int r = 0; r < C::RZ; ++r) {
                const int z = zrow0 + r;
                float2 l2[2], cc[2], inv[2] = {}, nom[2] = {}, o[2];
                f4(sL2 + (tz * C::RZ + r) * C::TX + 4 * tx, l2);
                f4(sC + (tz * C::RZ + r) * C::TX + 4 * tx, cc);
                if (rb < re) {
                    float2 src[2];
                    f4(ssrc + (tz * C::RZ + r) * C::TX + 4 * tx, src);
#pragma unroll
                    for (int h = 0; h < 2; ++h) Ll[r][h] = f2add(Ll[r][h], src[h]);
                }
                if constexpr (SP) sponge_row<C::RZ>(spr, r, inv, nom);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    o[h] = leapfrog<SP>(lc[r][h], l2[h], cc[h], Ll[r][h], inv[h], nom[h]);
                    if constexpr (!IMG64) acc[r][h] = f2fma(o[h], Qu[r][h], acc[r][h]);
                }
                if (z < p.g.NZ && xb < p.g.NX) st4(ln + (size_t)(z + GH) * p.g.P + (xb + GH), o, xb, p.g.NX);
                if constexpr (IMG64) {
                    if (z < p.g.NZ) {
                        double *im = p.img + ((size_t)(s / p.gsz) * p.k + j) * p.g.fsize + (size_t)(z + GH) * p.g.P +
                                     (xb + GH);
                        const float ov[4] = {o[0].x, o[0].y, o[1].x, o[1].y};
                        const float qv[4] = {Qu[r][0].x, Qu[r][0].y, Qu[r][1].x, Qu[r][1].y};
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (xb + c < p.g.NX) im[c] += (double)ov[c] * (double)qv[c];
                    }
                }
            }
            const bool group_end = (s + 1) % p.gsz == 0 || i + 1 == nitems;
            if (!IMG64 && group_end) flush(s / p.gsz);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (p.cnt && group_end) publish_item(p.cnt + (size_t)(s / p.gsz) * p.g.ntiles + tile);
                if (i + C::ST < nitems) issue(i + C::ST);
            }
        }
        return true;
    };
    if (sponge) run(std::true_type{});
    else run(std::false_type{});
}

// ------------------------------------------------------------------ resident kernels
// For grids whose padded field fits twice in one CTA's shared memory, H v with
// every forward level stored runs three persistent kernels instead of one
// launch per step: the forward field of each shot, and the Born field and the
// adjoint field of each (shot, vector) pair, stay in shared memory for all nt
// steps (zero initial and final conditions), so their only DRAM traffic is the
// per-step Q^n = Lh u^n + s_n (written once per shot, read by every pair), the
// coefficient fields and the receiver data.  Each thread owns blocks of 4 x 2
// points in a fixed order and computes them with the tiled kernels' exact
// arithmetic (lap_at, leapfrog, the Born source), so Q, the Born data and the
// adjoint fields are bitwise those of the tiled path; the image is accumulated
// per pair over all steps in double-float registers (each product split exactly)
// and the pairs' images are summed over shots in FP64 by the fold, an order
// that differs from the tiled path's per-step shot-group sums.
constexpr int kResNT = 480;      // threads per resident CTA (15 warps: 1352 blocks of the 104 x 104 grid spread ~2.8 each)
constexpr int kResRZ = 2;        // rows per thread block
constexpr int kResMaxB = 4;      // blocks per thread, upper bound
constexpr int kSmemCapResident = 227 * 1024;

struct ResParams {
    float *ws;                   // workspace base (field 0)
    int f_C, f_b, f_q;           // C, b [k], Q history: Q^n of shot s in field f_q + n ns + s
    float *dd;                   // Born data [k][ns][nt][nr]: written by the Born kernel, read by the adjoint
    float rscale;                // the adjoint source scale
    float2 *img;                 // per-pair images [ns][k][fsize], double-float (hi, lo)
    const float *az, *ax, *wavelet;
    const int *src_zx, *rt_rec, *rt_pos;
    int nt, nr, ns, k;
    int NZ, NX, P, W, nbx, nblocks;   // padded grid, global pitch, shared pitch NX + 8, blocks of 4 x 2
    unsigned long long fsize;
};

__device__ __forceinline__ void res_add_source(float2 (&Q)[kResRZ][2], int z0, int xb, int sz, int sx, float wav)
{
    const int dz = sz - z0, dx = sx - xb;
    if ((unsigned)dz < (unsigned)kResRZ && (unsigned)dx < 4u) {
#pragma unroll
        for (int r = 0; r < kResRZ; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (r == dz && c == dx) {
                    if (c & 1) Q[r][c >> 1].y += wav;
                    else Q[r][c >> 1].x += wav;
                }
    }
}

__device__ __forceinline__ size_t res_goff(const ResParams &p, int z, int xb)
{
    return (size_t)(z + GH) * p.P + (xb + GH);
}

// Shared memory of the resident kernels (floats): two fields [NZ + 9][W] (the
// padded field with its 4-cell ghost band and one spare row), then dense
// [NZ][NX] copies of the pointwise coefficients the kernel needs (C, and b or
// the image's low words), the damping profiles, and the adjoint's receiver
// tables.  Everything a step reads besides Q^n is on chip.  iz, ix = 1 / (1 +
// az), 1 / (1 + ax), correctly rounded; zt holds the row profile once more per
// pair of rows (the rows of one thread block) as (az, iz, az, iz), one 16-byte
// load per block.
struct ResSmem {
    float *F0, *F1, *C, *X, *az, *ax, *iz, *ix, *zt;
    int *tab;
};
static_assert(kResRZ == 2, "the row-profile table holds two rows per entry");
__device__ __forceinline__ ResSmem res_smem(const ResParams &p, float *base, bool second_dense)
{
    const int rowsW = (p.NZ + 2 * GH + 1) * p.W, N = p.NZ * p.NX;
    ResSmem m;
    m.F0 = base;
    m.F1 = base + rowsW;
    m.C = base + 2 * rowsW;
    m.X = m.C + N;
    const int NZ4 = (p.NZ + 3) & ~3;                 // keeps ax and ix 16-byte aligned (NX is a multiple of 4)
    m.zt = m.X + (second_dense ? N : 0);
    m.az = m.zt + 2 * NZ4;
    m.ax = m.az + NZ4;
    m.iz = m.ax + p.NX;
    m.ix = m.iz + NZ4;
    m.tab = reinterpret_cast<int *>(m.ix + p.NX);
    return m;
}

// Zero both fields, stage C (and `extra`, a [fsize] field, or zeros) densely, and the damping profiles.
__device__ __forceinline__ void res_setup(const ResParams &p, const ResSmem &m, const float *extra, bool second_dense)
{
    const int rowsW = (p.NZ + 2 * GH + 1) * p.W;
    for (int q = threadIdx.x; q < 2 * rowsW; q += kResNT) m.F0[q] = 0.0f;
    const float *C = p.ws + (unsigned long long)p.f_C * p.fsize;
    for (int q = threadIdx.x; q < p.NZ * p.NX; q += kResNT) {
        const int z = q / p.NX, x = q - z * p.NX;
        const size_t go = (size_t)(z + GH) * p.P + (x + GH);
        m.C[q] = C[go];
        if (second_dense) m.X[q] = extra ? extra[go] : 0.0f;
    }
    for (int q = threadIdx.x; q < p.NZ; q += kResNT) {
        m.az[q] = p.az[q];
        m.iz[q] = __frcp_rn(1.0f + p.az[q]);
    }
    for (int q = threadIdx.x; q < ((p.NZ + 3) & ~3); q += kResNT) {   // rows past NZ: a = 0
        const float a = q < p.NZ ? p.az[q] : 0.0f;
        m.zt[2 * q] = a;
        m.zt[2 * q + 1] = __frcp_rn(1.0f + a);
    }
    for (int q = threadIdx.x; q < p.NX; q += kResNT) {
        m.ax[q] = p.ax[q];
        m.ix[q] = __frcp_rn(1.0f + p.ax[q]);
    }
}

// The sponge factors of sponge_row from per-row and per-column tables: rounding
// is monotone, so 1 / (1 + max(az, ax)) rounded equals min(1 / (1 + az),
// 1 / (1 + ax)) rounded, and max(az, ax) - 1 equals max(az - 1, ax - 1):
// bitwise the values sponge_row computes, without a division per point.
// For the two rows z0, z0 + 1 (z0 even) of a thread block: three 16-byte loads
// per block (res_sponge_tabs), the factors of row r formed where they are used.
struct ResSpongeTabs {
    float4 z4, ix4, ax4;   // (az, iz) of both rows; ix and ax of the 4 columns
};

__device__ __forceinline__ ResSpongeTabs res_sponge_tabs(const ResSmem &m, int z0, int xb)
{
    return ResSpongeTabs{*reinterpret_cast<const float4 *>(m.zt + 2 * z0), *reinterpret_cast<const float4 *>(m.ix + xb),
                         *reinterpret_cast<const float4 *>(m.ax + xb)};
}

__device__ __forceinline__ void res_sponge_row(const ResSpongeTabs &t, int r, float2 (&inv)[2], float2 (&nom)[2])
{
    const float azv = r ? t.z4.z : t.z4.x, izv = r ? t.z4.w : t.z4.y;
    const float ixv[4] = {t.ix4.x, t.ix4.y, t.ix4.z, t.ix4.w}, axv[4] = {t.ax4.x, t.ax4.y, t.ax4.z, t.ax4.w};
    float iv[4], nm[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        iv[c] = fminf(izv, ixv[c]);
        nm[c] = fmaxf(azv, axv[c]) - 1.0f;
    }
    inv[0] = make_float2(iv[0], iv[1]);
    inv[1] = make_float2(iv[2], iv[3]);
    nom[0] = make_float2(nm[0], nm[1]);
    nom[1] = make_float2(nm[2], nm[3]);
}

// The same for one row z from the separate profiles (two 4-byte and two
// 16-byte loads; the adjoint has no registers to spare for a block's tables).
__device__ __forceinline__ void res_sponge_row_at(const ResSmem &m, int z, int xb, float2 (&inv)[2], float2 (&nom)[2])
{
    const float azv = m.az[z], izv = m.iz[z];
    res_sponge_row(ResSpongeTabs{make_float4(azv, izv, azv, izv), *reinterpret_cast<const float4 *>(m.ix + xb),
                                 *reinterpret_cast<const float4 *>(m.ax + xb)},
                   0, inv, nom);
}

__device__ __forceinline__ void res_block(const ResParams &p, int b, int &z0, int &xb, int &bx)
{
    const int bz = b / p.nbx;
    bx = b - bz * p.nbx;
    z0 = bz * kResRZ;
    xb = 4 * bx;
}

// The forward field of shot blockIdx.x: writes Q^n for n = 0 .. nt-1.
__global__ void __launch_bounds__(kResNT, 1) k_res_fwd(const __grid_constant__ ResParams p)
{
    extern __shared__ __align__(128) float rsm[];
    const ResSmem m = res_smem(p, rsm, false);
    res_setup(p, m, nullptr, false);
    const int s = blockIdx.x, sz = p.src_zx[2 * s], sx = p.src_zx[2 * s + 1];
    __syncthreads();
    for (int n = 0; n < p.nt; ++n) {
        const float *cur = (n & 1) ? m.F0 : m.F1;      // u^n
        float *prv = (n & 1) ? m.F1 : m.F0;            // u^{n-1}, overwritten by u^{n+1}
        const float wav = p.wavelet[n];
        float *qg = p.ws + (unsigned long long)(p.f_q + (long long)n * p.ns + s) * p.fsize;
        for (int b = threadIdx.x; b < p.nblocks; b += kResNT) {
            int z0, xb, bx;
            res_block(p, b, z0, xb, bx);
            float2 Q[kResRZ][2], uc[kResRZ][2];
            lap_at<kResRZ>(cur, p.W / 4, z0, bx + 1, Q, uc);
            res_add_source(Q, z0, xb, sz, sx, wav);
            const ResSpongeTabs spt = res_sponge_tabs(m, z0, xb);
#pragma unroll
            for (int r = 0; r < kResRZ; ++r) {
                const int z = z0 + r;
                if (z >= p.NZ) continue;
                *reinterpret_cast<float4 *>(qg + res_goff(p, z, xb)) =
                    make_float4(Q[r][0].x, Q[r][0].y, Q[r][1].x, Q[r][1].y);
                float2 up[2], cc[2], inv[2], nom[2], o[2];
                float *sp = prv + (z + GH) * p.W + xb + GH;
                f4(sp, up);
                f4(m.C + z * p.NX + xb, cc);
                res_sponge_row(spt, r, inv, nom);
#pragma unroll
                for (int h = 0; h < 2; ++h) o[h] = leapfrog<true>(uc[r][h], up[h], cc[h], Q[r][h], inv[h], nom[h]);
                *reinterpret_cast<float4 *>(sp) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
            }
        }
        __syncthreads();
    }
}

// Q^n at the thread's blocks, issued before the step's Laplacians so that the
// global loads overlap them.
template <int MAXB>
__device__ __forceinline__ void res_load_q(const ResParams &p, const float *qg, float4 (&qv)[MAXB][kResRZ])
{
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * kResNT;
        if (b >= p.nblocks) break;
        int z0, xb, bx;
        res_block(p, b, z0, xb, bx);
#pragma unroll
        for (int r = 0; r < kResRZ; ++r)
            qv[i][r] = z0 + r < p.NZ ? __ldg(reinterpret_cast<const float4 *>(qg + res_goff(p, z0 + r, xb)))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The Born field of pair (shot blockIdx.x, vector blockIdx.y): writes the Born data.
template <int MAXB>
__global__ void __launch_bounds__(kResNT, 1) k_res_born(const __grid_constant__ ResParams p)
{
    extern __shared__ __align__(128) float rsm[];
    const ResSmem m = res_smem(p, rsm, true);
    const int s = blockIdx.x, j = blockIdx.y;
    res_setup(p, m, p.ws + (unsigned long long)(p.f_b + j) * p.fsize, true);   // X = b_j
    float *dd = p.dd + ((size_t)j * p.ns + s) * p.nt * p.nr;
    __syncthreads();
    for (int n = 0; n < p.nt; ++n) {
        const float *cur = (n & 1) ? m.F0 : m.F1;      // du^n
        float *prv = (n & 1) ? m.F1 : m.F0;            // du^{n-1}, overwritten by du^{n+1}
        float4 qv[MAXB][kResRZ];
        res_load_q<MAXB>(p, p.ws + (unsigned long long)(p.f_q + (long long)n * p.ns + s) * p.fsize, qv);
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
            const int b = threadIdx.x + i * kResNT;
            if (b >= p.nblocks) break;
            int z0, xb, bx;
            res_block(p, b, z0, xb, bx);
            float2 Ld[kResRZ][2], dc[kResRZ][2];
            lap_at<kResRZ>(cur, p.W / 4, z0, bx + 1, Ld, dc);
            const ResSpongeTabs spt = res_sponge_tabs(m, z0, xb);
#pragma unroll
            for (int r = 0; r < kResRZ; ++r) {
                const int z = z0 + r;
                if (z >= p.NZ) continue;
                float2 dp[2], cc[2], bb[2], inv[2], nom[2], o[2];
                const float2 Q[2] = {lo(qv[i][r]), hi(qv[i][r])};
                float *sp = prv + (z + GH) * p.W + xb + GH;
                f4(sp, dp);
                f4(m.C + z * p.NX + xb, cc);
                f4(m.X + z * p.NX + xb, bb);
                res_sponge_row(spt, r, inv, nom);
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    o[h] = leapfrog<true>(dc[r][h], dp[h], cc[h], f2fma(bb[h], Q[h], Ld[r][h]), inv[h], nom[h]);
                *reinterpret_cast<float4 *>(sp) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < p.nr; q += kResNT) {   // du^{n+1} at the receivers
            const int pos = p.rt_pos[s * p.nr + q];
            const int z = pos / p.P - GH, x = pos - (pos / p.P) * p.P - GH;
            dd[(size_t)n * p.nr + p.rt_rec[s * p.nr + q]] = prv[(z + GH) * p.W + x + GH];
        }
    }
}

// The adjoint field of pair (shot blockIdx.x, vector blockIdx.y) and its image:
// the image's high words in registers, its low words in shared memory (X).
template <int MAXB>
__global__ void __launch_bounds__(kResNT, 1) k_res_adj(const __grid_constant__ ResParams p)
{
    extern __shared__ __align__(128) float rsm[];
    const ResSmem m = res_smem(p, rsm, true);
    res_setup(p, m, nullptr, true);                   // X = 0: the image's low words
    int *cnt = m.tab;                                 // [nblocks + 1]: receivers per block, then starts
    int *fill = cnt + p.nblocks + 1;                  // [nblocks]
    int *ent = fill + p.nblocks;                      // [nr]: (lane << 16) | receiver slot q
    for (int q = threadIdx.x; q <= p.nblocks; q += kResNT) cnt[q] = 0;
    for (int q = threadIdx.x; q < p.nblocks; q += kResNT) fill[q] = 0;
    const int s = blockIdx.x, j = blockIdx.y;
    __syncthreads();
    // receivers of the shot by thread block (a block holds at most one receiver per point)
    auto rec_block = [&](int q, int &lane) {
        const int pos = p.rt_pos[s * p.nr + q];
        const int z = pos / p.P - GH, x = pos - (pos / p.P) * p.P - GH;
        lane = (z % kResRZ) * 4 + (x & 3);
        return (z / kResRZ) * p.nbx + (x >> 2);
    };
    for (int q = threadIdx.x; q < p.nr; q += kResNT) {
        int lane;
        atomicAdd(&cnt[rec_block(q, lane) + 1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < p.nblocks; ++b) cnt[b + 1] += cnt[b];
    __syncthreads();
    for (int q = threadIdx.x; q < p.nr; q += kResNT) {
        int lane;
        const int b = rec_block(q, lane);
        ent[cnt[b] + atomicAdd(&fill[b], 1)] = (lane << 16) | q;
    }
    const float *rs0 = p.dd + ((size_t)j * p.ns + s) * p.nt * p.nr;
    float4 hi4[MAXB][kResRZ];
#pragma unroll
    for (int i = 0; i < MAXB; ++i)
#pragma unroll
        for (int r = 0; r < kResRZ; ++r) hi4[i][r] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    // (h, l) += a exactly-split product: TwoSum of the rounded product, its rounding error to l
    auto acc = [](float &h_, float &l_, float o, float q) {
        const float pr = __fmul_rn(o, q), pe = fmaf(o, q, -pr);
        const float t = __fadd_rn(h_, pr), bv = __fsub_rn(t, h_);
        l_ = __fadd_rn(l_, __fadd_rn(__fadd_rn(__fsub_rn(h_, __fsub_rn(t, bv)), __fsub_rn(pr, bv)), pe));
        h_ = t;
    };
    for (int mstep = 0; mstep < p.nt; ++mstep) {
        const int n = p.nt - 1 - mstep;
        const float *cur = (mstep & 1) ? m.F0 : m.F1;   // lambda^{n+1}
        float *prv = (mstep & 1) ? m.F1 : m.F0;         // lambda^{n+2}, overwritten by lambda^n
        const float *rs = rs0 + (size_t)n * p.nr;
        float4 qv[MAXB][kResRZ];
        res_load_q<MAXB>(p, p.ws + (unsigned long long)(p.f_q + (long long)n * p.ns + s) * p.fsize, qv);
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
            const int b = threadIdx.x + i * kResNT;
            if (b >= p.nblocks) break;
            int z0, xb, bx;
            res_block(p, b, z0, xb, bx);
            float2 Ll[kResRZ][2], lc[kResRZ][2];
            lap_at<kResRZ>(cur, p.W / 4, z0, bx + 1, Ll, lc);
            for (int e = cnt[b]; e < cnt[b + 1]; ++e) {          // receiver sources: added to Lh lambda
                const int lane = ent[e] >> 16, q = ent[e] & 0xffff;
                const float v = p.rscale * rs[p.rt_rec[s * p.nr + q]];
                float2 &t = Ll[lane >> 2][(lane & 3) >> 1];
                if (lane & 1) t.y = __fadd_rn(t.y, v);
                else t.x = __fadd_rn(t.x, v);
            }
#pragma unroll
            for (int r = 0; r < kResRZ; ++r) {
                const int z = z0 + r;
                if (z >= p.NZ) continue;
                float2 l2[2], cc[2], inv[2], nom[2], o[2];
                float *sp = prv + (z + GH) * p.W + xb + GH;
                f4(sp, l2);
                f4(m.C + z * p.NX + xb, cc);
                res_sponge_row_at(m, z, xb, inv, nom);
#pragma unroll
                for (int h = 0; h < 2; ++h) o[h] = leapfrog<true>(lc[r][h], l2[h], cc[h], Ll[r][h], inv[h], nom[h]);
                *reinterpret_cast<float4 *>(sp) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                // image += lambda^n Q^n (double-float: high words here, low words in shared memory)
                float4 *lw = reinterpret_cast<float4 *>(m.X + z * p.NX + xb);
                float4 l4 = *lw;
                float4 &h4 = hi4[i][r];
                const float4 q4 = qv[i][r];
                acc(h4.x, l4.x, o[0].x, q4.x);
                acc(h4.y, l4.y, o[0].y, q4.y);
                acc(h4.z, l4.z, o[1].x, q4.z);
                acc(h4.w, l4.w, o[1].y, q4.w);
                *lw = l4;
            }
        }
        __syncthreads();
    }
    float2 *im = p.img + ((size_t)s * p.k + j) * p.fsize;
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * kResNT;
        if (b >= p.nblocks) break;
        int z0, xb, bx;
        res_block(p, b, z0, xb, bx);
#pragma unroll
        for (int r = 0; r < kResRZ; ++r) {
            const int z = z0 + r;
            if (z >= p.NZ) continue;
            float2 *q = im + res_goff(p, z, xb);
            const float4 h4 = hi4[i][r], l4 = *reinterpret_cast<const float4 *>(m.X + z * p.NX + xb);
            reinterpret_cast<float4 *>(q)[0] = make_float4(h4.x, l4.x, h4.y, l4.y);
            reinterpret_cast<float4 *>(q)[1] = make_float4(h4.z, l4.z, h4.w, l4.w);
        }
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int encode(void *map, const hv_handle *h, void *ws, long long nfields, int boxx, int boxz)
{
    auto fn = encode_fn();
    if (!fn) return hvi::fail(HV_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {(cuuint64_t)h->P, (cuuint64_t)h->rows, (cuuint64_t)nfields};
    cuuint64_t strides[2] = {(cuuint64_t)h->P * 4, (cuuint64_t)h->fsize * 4};
    cuuint32_t box[3] = {(cuuint32_t)boxx, (cuuint32_t)boxz, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ws, dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hvi::fail(HV_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HV_OK;
}

int field_index(const void *ws, const void *p, size_t fbytes, int *out)
{
    if (!p) {
        *out = -1;
        return HV_OK;
    }
    ptrdiff_t d = (const char *)p - (const char *)ws;
    if (d < 0 || (size_t)d % fbytes != 0) return hvi::fail(HV_EINVAL, "internal: field not aligned in the workspace");
    *out = (int)((size_t)d / fbytes);
    return HV_OK;
}

// Calls f with a value of the tile configuration `id` (see kTileMenu).
template <class F>
auto with_cfg(int id, F &&f)
{
    switch (id) {
    case 1: return f(Cfg32x32{});
    case 2: return f(Cfg64x16{});
    case 3: return f(Cfg52x26{});
    case 4: return f(Cfg128x16{});
    case 5: return f(Cfg64x8{});
    case 6: return f(Cfg32x16{});
    case 7: return f(Cfg128x8{});
    case 8: return f(Cfg32x16s3{});
    case 9: return f(Cfg32x16g4{});
    case 10: return f(Cfg32x16s3g4{});
    case 11: return f(Cfg128x8s3{});
    case 12: return f(Cfg128x8g4{});
    case 13: return f(Cfg128x8s3g4{});
    case 14: return f(Cfg64x16s3g2{});
    case 15: return f(Cfg64x8s3g4{});
    default: return f(Cfg64x32{});
    }
}

template <class K>
int set_smem(K kern, int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return HV_OK;
}

// Raise a kernel's dynamic shared memory limit once per (kernel, device).
template <class K>
int ensure_smem(int slot, int dev, K kern, int bytes)
{
    static std::mutex mu;
    static bool done[96][64] = {};
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 96) return hvi::fail(HV_EINVAL, "internal: kernel slot %d/%d", slot, dev);
    std::lock_guard<std::mutex> g(mu);
    if (done[slot][dev]) return HV_OK;
    HV_RT_INTERNAL(set_smem(kern, bytes));
    done[slot][dev] = true;
    return HV_OK;
}

// Launches a stencil step, with programmatic dependent launch when enabled.
template <class P>
int launch_step(void (*kern)(P), dim3 grid, int threads, int smem, cudaStream_t st, bool pdl, const P &p,
                const char *what)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = pdl ? 1 : 0;
    count_launch();
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, p);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

bool pdl(const hv_handle *h) { return h->launch_mode >= HV_LAUNCH_PDL; }

Geo geo(const hv_handle *h, const hvi::Tiling &t)
{
    return Geo{h->P, h->NZ, h->NX, h->nz, h->nx, h->nb, t.ntx, t.ntiles, (unsigned long long)h->fsize};
}

}  // namespace

int tile_menu_size() { return kTileMenu; }

int max_tiles(const hv_handle *h)
{
    int m = 0;
    for (int c = 0; c < kTileMenu; ++c) m = std::max(m, tiling(h, c).ntiles);
    return m;
}

void menu_info(int cfg, int *info)
{
    with_cfg(cfg, [&](auto c) {
        using C = decltype(c);
        info[0] = C::TX;
        info[1] = C::TZ;
        info[2] = C::NT;
        info[3] = C::ST;
        info[4] = C::GPC;
        return 0;
    });
}

hvi::Tiling tiling(const hv_handle *h, int cfg)
{
    return with_cfg(cfg, [&](auto c) {
        using C = decltype(c);
        hvi::Tiling t;
        t.TX = C::TX;
        t.TZ = C::TZ;
        t.ntx = (h->NX + C::TX - 1) / C::TX;
        t.ntz = (h->NZ + C::TZ - 1) / C::TZ;
        t.ntiles = t.ntx * t.ntz;
        return t;
    });
}

// Shot groups of the adjoint kernel: G = ceil(ns / 8) groups of ceil(ns / G)
// consecutive shots, each summed in FP32 in shot order per step and added to
// its own double-float partial image; the partials are summed in group order at the
// end.  The grouping depends only on the shot count (never on k, the tile
// shape or how many groups a CTA walks), so a vector's result is bitwise the
// same whether it is applied alone or in a batch.
int adj_groups(const hv_handle *h) { return (h->ns + kShotsPerGroup - 1) / kShotsPerGroup; }

// Raise the shared-memory limits of every stencil kernel on the handle's
// device (done at set-up so that no attribute call happens during capture).
int prepare_kernels(const hv_handle *h)
{
    for (int id = 0; id < kTileMenu; ++id) {
        int rc = with_cfg(id, [&](auto c) -> int {
            using C = decltype(c);
            HV_RT_INTERNAL(ensure_smem(0 * kTileMenu + id, h->device, k_fwd<C, true>, FwdSmem<C, true>::BYTES));
            HV_RT_INTERNAL(ensure_smem(1 * kTileMenu + id, h->device, k_fwd<C, false>, FwdSmem<C, false>::BYTES));
            HV_RT_INTERNAL(ensure_smem(2 * kTileMenu + id, h->device, k_adj<C>, AdjSmem<C>::BYTES));
            HV_RT_INTERNAL(ensure_smem(3 * kTileMenu + id, h->device, k_fwd2<C>, Fwd2Smem<C>::BYTES));
            return HV_OK;
        });
        if (rc != HV_OK) return rc;
    }
    return ensure_smem(4 * kTileMenu, h->device, k_adj<Cfg64x8, true>, AdjSmem<Cfg64x8>::BYTES);
}

int adj_f64_cfg() { return 5; }   // the menu entry (64 x 8) that has the FP64-image adjoint

int make_maps(const hv_handle *h, void *ws, long long nfields, TmaMaps *m)
{
    for (int id = 0; id < kTileMenu; ++id) {
        int rc = with_cfg(id, [&](auto c) {
            using C = decltype(c);
            HV_RT_INTERNAL(encode(m->halo[id], h, ws, nfields, C::W, C::H));
            HV_RT_INTERNAL(encode(m->pt[id], h, ws, nfields, C::TX, C::TZ));
            HV_RT_INTERNAL(encode(m->halo8[id], h, ws, nfields, C::TX + 16, C::TZ + 16));
            return (int)HV_OK;
        });
        if (rc != HV_OK) return rc;
    }
    m->ws = ws;
    m->nfields = nfields;
    return HV_OK;
}

int launch_fwd(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const FwdLaunch &a,
               cudaStream_t st)
{
    return with_cfg(cfg, [&](auto c) -> int {
        using C = decltype(c);
        const hvi::Tiling t = tiling(h, cfg);
        const size_t fbytes = h->fsize * sizeof(float);
        FwdParams p;
        memcpy(&p.map_halo, maps.halo[cfg], sizeof(CUtensorMap));
        memcpy(&p.map_pt, maps.pt[cfg], sizeof(CUtensorMap));
        p.ws = reinterpret_cast<float *>(maps.ws);
        HV_RT_INTERNAL(field_index(maps.ws, a.u_cur, fbytes, &p.f_ucur));
        HV_RT_INTERNAL(field_index(maps.ws, a.u_prev, fbytes, &p.f_uprev));
        HV_RT_INTERNAL(field_index(maps.ws, a.u_next, fbytes, &p.f_unext));
        HV_RT_INTERNAL(field_index(maps.ws, a.C, fbytes, &p.f_C));
        const bool born = a.b != nullptr && a.k > 0;
        if (!born && a.models > 1 && a.deps.cnt)
            return hvi::fail(HV_EINVAL, "internal: step counters with %d models in one launch", a.models);
        HV_RT_INTERNAL(field_index(maps.ws, born ? a.b : nullptr, fbytes, &p.f_b));
        HV_RT_INTERNAL(field_index(maps.ws, born ? a.du_cur : nullptr, fbytes, &p.f_du));
        HV_RT_INTERNAL(field_index(maps.ws, born ? a.du_io : nullptr, fbytes, &p.f_dio));
        p.d_u = a.d_u;
        p.d_du = born ? a.d_du : nullptr;
        p.slot_join = born ? nullptr : a.slot_join;
        p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
        p.src_zx = h->src_zx; p.rt_off = rt.off; p.rt_rec = rt.rec; p.rt_pos = rt.pos;
        p.status = h->status;
        p.wait_ns = h->wait_ns;
        p.n = a.n; p.nt = h->nt; p.nr = h->nr; p.ns = h->ns; p.k = born ? a.k : std::max(a.models, 1);
        p.gsz = (h->ns + adj_groups(h) - 1) / adj_groups(h);   // the adjoint's shot groups
        p.spg = p.gsz * C::GPC;                                  // shots per CTA: GPC whole groups
        p.cnt = a.deps.cnt;
        p.need = a.deps.need;
        p.flow = a.deps.flow ? 1 : 0;
        p.g = geo(h, t);
        dim3 grid(t.ntiles, p.k, (h->ns + p.spg - 1) / p.spg);
        if (born) {
            HV_RT_INTERNAL(ensure_smem(0 * kTileMenu + cfg, h->device, k_fwd<C, true>, FwdSmem<C, true>::BYTES));
            return launch_step(k_fwd<C, true>, grid, C::NT, FwdSmem<C, true>::BYTES, st, pdl(h), p, "k_fwd launch");
        }
        HV_RT_INTERNAL(ensure_smem(1 * kTileMenu + cfg, h->device, k_fwd<C, false>, FwdSmem<C, false>::BYTES));
        return launch_step(k_fwd<C, false>, grid, C::NT, FwdSmem<C, false>::BYTES, st, pdl(h) && !a.plain, p,
                           "k_fwd launch");
    });
}

int fwd_ctas_per_model(const hv_handle *h, int cfg)
{
    return with_cfg(cfg, [&](auto c) -> int {
        using C = decltype(c);
        const int gsz = (h->ns + adj_groups(h) - 1) / adj_groups(h), spg = gsz * C::GPC;
        return tiling(h, cfg).ntiles * ((h->ns + spg - 1) / spg);
    });
}

int launch_fwd2(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const Fwd2Launch &a,
                cudaStream_t st)
{
    if (a.n + 1 >= h->nt) return hvi::fail(HV_EINVAL, "internal: fused steps %d, %d past nt = %d", a.n, a.n + 1, h->nt);
    return with_cfg(cfg, [&](auto c) -> int {
        using C = decltype(c);
        const hvi::Tiling t = tiling(h, cfg);
        const size_t fbytes = h->fsize * sizeof(float);
        Fwd2Params p;
        memcpy(&p.map_halo, maps.halo[cfg], sizeof(CUtensorMap));
        memcpy(&p.map_halo8, maps.halo8[cfg], sizeof(CUtensorMap));
        p.ws = reinterpret_cast<float *>(maps.ws);
        HV_RT_INTERNAL(field_index(maps.ws, a.u_cur, fbytes, &p.f_ucur));
        HV_RT_INTERNAL(field_index(maps.ws, a.u_prev, fbytes, &p.f_uprev));
        HV_RT_INTERNAL(field_index(maps.ws, a.u_next1, fbytes, &p.f_unext1));
        HV_RT_INTERNAL(field_index(maps.ws, a.u_next2, fbytes, &p.f_unext2));
        HV_RT_INTERNAL(field_index(maps.ws, a.C, fbytes, &p.f_C));
        if (p.f_unext1 < 0 || p.f_unext2 < 0 || p.f_unext1 == p.f_unext2 || p.f_unext1 == p.f_ucur ||
            p.f_unext1 == p.f_uprev || p.f_unext2 == p.f_ucur || p.f_unext2 == p.f_uprev)
            return hvi::fail(HV_EINVAL, "internal: fused steps need two outputs distinct from the inputs");
        p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
        p.src_zx = h->src_zx; p.rt_off = rt.off;
        p.status = h->status;
        p.wait_ns = h->wait_ns;
        p.n = a.n; p.ns = h->ns;
        const int gsz = (h->ns + adj_groups(h) - 1) / adj_groups(h);
        p.spg = gsz * C::GPC;
        p.g = geo(h, t);
        dim3 grid(t.ntiles, 1, (h->ns + p.spg - 1) / p.spg);
        HV_RT_INTERNAL(ensure_smem(3 * kTileMenu + cfg, h->device, k_fwd2<C>, Fwd2Smem<C>::BYTES));
        return launch_step(k_fwd2<C>, grid, C::NT, Fwd2Smem<C>::BYTES, st, pdl(h), p, "k_fwd2 launch");
    });
}

// ------------------------------------------------------------------ resident path (host)
namespace {
struct ResGeo {
    int W, nbx, nblocks, maxb;
    size_t smem_fwd, smem_born, smem_adj;
};
int res_launched(const char *what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return HV_OK;
}

ResGeo res_geo(const hv_handle *h)
{
    ResGeo g;
    g.W = h->NX + 2 * GH;
    g.nbx = h->NX / 4;
    g.nblocks = g.nbx * ((h->NZ + kResRZ - 1) / kResRZ);
    g.maxb = (g.nblocks + kResNT - 1) / kResNT;
    const size_t field = (size_t)(h->NZ + 2 * GH + 1) * g.W * sizeof(float);
    const size_t dense = (size_t)h->NZ * h->NX * sizeof(float),
                 prof = (4 * (size_t)((h->NZ + 3) & ~3) + 2 * (size_t)h->NX) * sizeof(float);   // ResSmem profiles
    g.smem_fwd = 2 * field + dense + prof;                       // fields, C, profiles
    g.smem_born = 2 * field + 2 * dense + prof;                  // + b_j
    g.smem_adj = 2 * field + 2 * dense + prof + (size_t)(2 * g.nblocks + 1 + h->nr) * sizeof(int);   // + image low words, tables
    return g;
}
}  // namespace

bool resident_fits(const hv_handle *h)
{
    if (h->NX % 4 != 0 || h->nr >= 65536) return false;
    const ResGeo g = res_geo(h);
    return g.maxb >= 1 && g.maxb <= kResMaxB && g.smem_adj <= (size_t)kSmemCapResident;
}

int launch_resident(const hv_handle *h, int which, const ResLaunch &a, cudaStream_t st)
{
    if (!resident_fits(h)) return hvi::fail(HV_EINVAL, "internal: the grid does not fit the resident kernels");
    const ResGeo g = res_geo(h);
    const size_t fbytes = h->fsize * sizeof(float);
    ResParams p;
    p.ws = reinterpret_cast<float *>(a.base);
    HV_RT_INTERNAL(field_index(a.base, a.C, fbytes, &p.f_C));
    HV_RT_INTERNAL(field_index(a.base, a.b, fbytes, &p.f_b));
    HV_RT_INTERNAL(field_index(a.base, a.q, fbytes, &p.f_q));
    p.dd = a.dd;
    p.rscale = a.rscale;
    p.img = reinterpret_cast<float2 *>(a.img);
    p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
    p.src_zx = h->src_zx; p.rt_rec = a.rec; p.rt_pos = a.pos;
    p.nt = h->nt; p.nr = h->nr; p.ns = h->ns; p.k = a.k;
    p.NZ = h->NZ; p.NX = h->NX; p.P = h->P; p.W = g.W; p.nbx = g.nbx; p.nblocks = g.nblocks;
    p.fsize = h->fsize;
    static std::mutex mu;
    static bool attr[64][1 + 2 * kResMaxB] = {};
    auto prep = [&](auto kern, int slot, size_t bytes) -> int {
        std::lock_guard<std::mutex> lk(mu);
        if (h->device < 0 || h->device >= 64) return hvi::fail(HV_EINVAL, "internal: device %d", h->device);
        if (!attr[h->device][slot]) {
            HV_RT_INTERNAL(set_smem(kern, kSmemCapResident));
            attr[h->device][slot] = true;
        }
        (void)bytes;
        return HV_OK;
    };
    if (which == 0) {
        HV_RT_INTERNAL(prep(k_res_fwd, 0, g.smem_fwd));
        k_res_fwd<<<h->ns, kResNT, g.smem_fwd, st>>>(p);
        return res_launched("k_res_fwd launch");
    }
    auto pair = [&](auto kern, int slot, size_t bytes, const char *what) -> int {
        HV_RT_INTERNAL(prep(kern, slot, bytes));
        kern<<<dim3(h->ns, a.k), kResNT, bytes, st>>>(p);
        return res_launched(what);
    };
    const int mb = std::min(g.maxb, kResMaxB);
    if (which == 1) {
        switch (mb) {
        case 1: return pair(k_res_born<1>, 1, g.smem_born, "k_res_born launch");
        case 2: return pair(k_res_born<2>, 2, g.smem_born, "k_res_born launch");
        case 3: return pair(k_res_born<3>, 3, g.smem_born, "k_res_born launch");
        default: return pair(k_res_born<4>, 4, g.smem_born, "k_res_born launch");
        }
    }
    switch (mb) {
    case 1: return pair(k_res_adj<1>, 5, g.smem_adj, "k_res_adj launch");
    case 2: return pair(k_res_adj<2>, 6, g.smem_adj, "k_res_adj launch");
    case 3: return pair(k_res_adj<3>, 7, g.smem_adj, "k_res_adj launch");
    default: return pair(k_res_adj<4>, 8, g.smem_adj, "k_res_adj launch");
    }
}

int launch_adj(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const AdjLaunch &a,
               cudaStream_t st)
{
    return with_cfg(cfg, [&](auto c) -> int {
        using C = decltype(c);
        const hvi::Tiling t = tiling(h, cfg);
        const size_t fbytes = h->fsize * sizeof(float);
        AdjParams p;
        memcpy(&p.map_halo, maps.halo[cfg], sizeof(CUtensorMap));
        memcpy(&p.map_pt, maps.pt[cfg], sizeof(CUtensorMap));
        p.ws = reinterpret_cast<float *>(maps.ws);
        HV_RT_INTERNAL(field_index(maps.ws, a.u, fbytes, &p.f_u));
        HV_RT_INTERNAL(field_index(maps.ws, a.lam1, fbytes, &p.f_lam1));
        HV_RT_INTERNAL(field_index(maps.ws, a.lam_io, fbytes, &p.f_lamio));
        HV_RT_INTERNAL(field_index(maps.ws, a.C, fbytes, &p.f_C));
        p.r = a.r;
        p.r_vstride = a.r_per_vector ? (unsigned long long)h->ns * h->nt * h->nr : 0ull;
        p.rscale = a.rscale;
        p.img = a.img;
        p.az = h->az; p.ax = h->ax; p.wavelet = h->wavelet;
        p.src_zx = h->src_zx; p.rt_off = rt.off; p.rt_rec = rt.rec; p.rt_pos = rt.pos;
        p.status = h->status;
        p.wait_ns = h->wait_ns;
        p.n = a.n; p.nt = h->nt; p.nr = h->nr; p.ns = h->ns; p.k = a.k;
        p.gsz = (h->ns + a.G - 1) / a.G;    // shots per group (the last group may be shorter)
        p.spg = p.gsz * C::GPC;             // shots per CTA: GPC whole groups
        p.cnt = a.deps.cnt;
        p.need = a.deps.need;
        p.flow = a.deps.flow ? 1 : 0;
        p.g = geo(h, t);
        dim3 grid(t.ntiles, a.k, (a.G + C::GPC - 1) / C::GPC);
        if constexpr (std::is_same<C, Cfg64x8>::value) {
            if (a.img_f64) {
                HV_RT_INTERNAL(ensure_smem(4 * kTileMenu, h->device, k_adj<C, true>, AdjSmem<C>::BYTES));
                return launch_step(k_adj<C, true>, grid, C::NT, AdjSmem<C>::BYTES, st, pdl(h), p, "k_adj launch");
            }
        }
        HV_RT_INTERNAL(ensure_smem(2 * kTileMenu + cfg, h->device, k_adj<C>, AdjSmem<C>::BYTES));
        return launch_step(k_adj<C>, grid, C::NT, AdjSmem<C>::BYTES, st, pdl(h), p, "k_adj launch");
    });
}

}  // namespace hvk
