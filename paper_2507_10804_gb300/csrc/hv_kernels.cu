// hv_kernels.cu -- the non-stencil kernels of the Gauss-Newton Hessian apply:
// model preparation, image fold, misfit reduction, set-up and housekeeping
// (the time-stepping kernels are in hv_stencil.cu).
//
// The stencil coefficients, the sponge and the time-stepping identities they
// serve are described in hv_stencil.cu.  Here: C = (m dt / h)^2 and the Born
// coefficient b = 2 (E v) / (E m) on the padded grid (the model and vectors
// are replicated into the sponge by E), the sponge rates a = q dt / 2 per
// axis and the Ricker wavelet, the fold Hv = E^T ((2 / (m h^2)) image), the
// FP64 misfit reduction, the ghost-band clearing and the wavefield export.
#include "hv_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>

namespace hvk {

using hvi::GH;

namespace {

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

// The image of group g, vector j at padded node offset `off` in format fmt:
// 0: double-float (hi, lo) FP32 pairs per group in the field layout, 1: FP64
// per group in the field layout, 2: one dense FP64 image [k][NZ][NX] (g = 0).
__device__ __forceinline__ double img_at(const double *img, int fmt, int g, int k, int j, size_t fsize, size_t off,
                                         int z, int x, int NZ, int NX)
{
    if (fmt == 0) {
        const float2 v = reinterpret_cast<const float2 *>(img)[((size_t)g * k + j) * fsize + off];
        return (double)v.x + (double)v.y;
    }
    if (fmt == 1) return img[((size_t)g * k + j) * fsize + off];
    return img[((size_t)j * NZ + z) * NX + x];
}

// The fold Hv[j][iz][ix] = 2 / (m h^2) * (E^T sum_g img_g)[iz][ix] in three
// passes, so that no thread walks more than one group list or one sponge
// width (a 41 x 41 corner of 4 groups on the benchmark's grid, of 32 per-pair
// images on the resident path, took one thread 1-2 ms): k_fold_g sums the
// groups of every padded node in group order in FP64 and writes the sum over
// group 0's word of that node (each thread reads and writes its own node
// only); k_fold_x sums the x-preimage of each interior column of every padded
// row into t[j][z][ix]; k_fold_z sums the z-preimage of each interior row of t
// and scales.
__global__ void k_fold_g(double *img, int fmt, int G, int k, int NZ, int NX, int P, size_t fsize)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y, j = blockIdx.z;
    if (x >= NX) return;
    const size_t off = (size_t)(z + GH) * P + (x + GH);
    double acc = 0.0;
    for (int g = 0; g < G; ++g) acc += img_at(img, fmt, g, k, j, fsize, off, z, x, NZ, NX);
    img[(size_t)j * fsize + off] = acc;
}

__global__ void k_fold_x(const double *__restrict__ gsum, int nx, int nb, int NZ, int NX, int P, size_t fsize,
                         double *__restrict__ t)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int j = blockIdx.z;
    if (ix >= nx) return;
    const int xlo = (ix == 0) ? 0 : ix + nb, xhi = (ix == nx - 1) ? NX - 1 : ix + nb;
    double acc = 0.0;
    for (int x = xlo; x <= xhi; ++x) acc += gsum[(size_t)j * fsize + (size_t)(z + GH) * P + (x + GH)];
    t[((size_t)j * NZ + z) * nx + ix] = acc;
}

__global__ void k_fold_z(const float *__restrict__ m, const double *__restrict__ t, int nz, int nx, int nb, int NZ,
                         double h, float *out32, double *out64)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int j = blockIdx.z;
    if (ix >= nx) return;
    const int zlo = (iz == 0) ? 0 : iz + nb, zhi = (iz == nz - 1) ? NZ - 1 : iz + nb;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z) acc += t[((size_t)j * NZ + z) * nx + ix];
    const double mm = (double)m[(size_t)iz * nx + ix];
    const double val = 2.0 / (mm * h * h) * acc;
    const size_t o = ((size_t)j * nz + iz) * nx + ix;
    if (out32) out32[o] = (float)val;
    if (out64) out64[o] = val;
}

// The extended image of this handle's shots on the padded grid (before the
// fold E^T): out[j][z][x] = 2 / (m_ext h^2) * sum_g img_g, the groups summed
// in group order in FP64, m_ext = E m (the nearest interior value).
__global__ void k_partial_image(const float *__restrict__ m, const double *__restrict__ img, int fmt, int G, int k,
                                int nz, int nx, int nb, int NZ, int NX, int P, size_t fsize, double h,
                                double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y, j = blockIdx.z;
    if (x >= NX) return;
    const size_t off = (size_t)(z + GH) * P + (x + GH);
    double acc = 0.0;
    for (int g = 0; g < G; ++g) acc += img_at(img, fmt, g, k, j, fsize, off, z, x, NZ, NX);
    const int iz = min(max(z - nb, 0), nz - 1), ix = min(max(x - nb, 0), nx - 1);
    const double mm = (double)m[(size_t)iz * nx + ix];
    out[((size_t)j * NZ + z) * NX + x] = 2.0 / (mm * h * h) * acc;
}

// The fold E^T of extended images ext[k][NZ][NX] (FP64) onto the interior:
// every sponge node adds onto its nearest interior node.
__global__ void k_fold_ext(const double *__restrict__ ext, int nz, int nx, int nb, int NZ, int NX, float *out32,
                           double *out64)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y, j = blockIdx.z;
    if (ix >= nx) return;
    const int zlo = (iz == 0) ? 0 : iz + nb, zhi = (iz == nz - 1) ? NZ - 1 : iz + nb;
    const int xlo = (ix == 0) ? 0 : ix + nb, xhi = (ix == nx - 1) ? NX - 1 : ix + nb;
    double acc = 0.0;
    for (int z = zlo; z <= zhi; ++z)
        for (int x = xlo; x <= xhi; ++x) acc += ext[((size_t)j * NZ + z) * NX + x];
    const size_t o = ((size_t)j * nz + iz) * nx + ix;
    if (out32) out32[o] = (float)acc;
    if (out64) out64[o] = acc;
}

// Block `blk` of `nblk` of the residual r = d - d_obs and its FP64 sum of
// squares: a grid stride over n, then a fixed warp-shuffle tree (fixed
// assignment, fixed tree: the value depends only on n, nblk and the block
// size, never on which kernel runs the block).
__device__ __forceinline__ void residual_block(const float *d, const float *__restrict__ dobs, float *r, size_t n,
                                               double *__restrict__ partials, int blk, int nblk)
{
    __shared__ double sw[32];
    double acc = 0.0;
    for (size_t i = (size_t)blk * blockDim.x + threadIdx.x; i < n; i += (size_t)nblk * blockDim.x) {
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
        if (threadIdx.x == 0) partials[blk] = v;
    }
}

// phi = scale * (the nb partials summed by one block in a fixed tree).
__device__ __forceinline__ void reduce_partials(const double *__restrict__ partials, int nb, double scale, double *phi)
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

// r = d - dobs and per-block FP64 partial sums of r^2.
__global__ void k_residual(const float *d, const float *__restrict__ dobs, float *r, size_t n,
                           double *__restrict__ partials)
{
    residual_block(d, dobs, r, n, partials, blockIdx.x, gridDim.x);
}


__global__ void k_reduce_phi(const double *__restrict__ partials, int nb, double scale, double *phi)
{
    reduce_partials(partials, nb, scale, phi);
}

// Adds the number of non-finite entries (NaN or +-Inf) of x[0, n) to *count.
__global__ void k_count_nonfinite(const float *__restrict__ x, size_t n, unsigned long long *count)
{
    unsigned c = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += !isfinite(x[i]);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// ---- the device-resident misfit loop (one iteration of its graph body per time step)

// Admission and step bookkeeping of every slot (one block).  After a step
// (after_tick): the slots that took their last step are listed for the misfit
// kernels and freed, and every other occupied slot advances; then (in both
// modes) a free slot whose mailbox holds a new sequence number is admitted at
// step 0 (its model and fields were prepared before the number was posted),
// the step table of the next step is written for k_fwd, and the conditions
// are set: another iteration or not, which step launch comes next (the
// smallest power-of-two prefix of slots covering the highest occupied one, or
// the body without a step), and whether this iteration's misfit kernels run.
// Launched behind the step by programmatic dependent launch: it is resident
// while the step drains and waits for it before touching the tables.
__global__ void k_loop_control(const LoopParams p)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ int occ, ymax;
    if (threadIdx.x == 0) {
        occ = ymax = 0;
        int nf = 0;                            // in slot order (one thread: the list is short, its order fixed)
        if (p.after_tick)
            for (int j = 0; j < p.slots; ++j)
                if (p.step[j] == p.nt - 1) p.fin[nf++] = j;
        p.fin[p.slots] = nf;
    }
    __syncthreads();
    int local = 0, top = 0;
    for (int j = threadIdx.x; j < p.slots; j += blockDim.x) {
        int st = p.step[j];
        if (p.after_tick && st >= 0 && ++st >= p.nt) st = -1;
        const int posted = *reinterpret_cast<volatile const int *>(p.post + j);
        if (st < 0 && posted != p.seen[j]) {
            __threadfence();                   // the request's prepared fields, written before the post
            st = 0;
            p.seen[j] = posted;
            p.ack[j] = posted;
        }
        p.step[j] = st;
        p.join[j] = st >= 0 ? -st : kLoopFreeSlot;
        local += st >= 0;
        if (st >= 0) top = j + 1;
    }
    atomicAdd(&occ, local);
    atomicMax(&ymax, top);
    __syncthreads();
    // The loop goes on unless the host asked it to stop, max_iter iterations of
    // this launch have run, or no slot has been occupied for idle_max
    // iterations (a request posted after this scan is admitted by the next launch).
    if (threadIdx.x == 0) {
        p.ctl[2] = occ;
        const int it = p.ctl[0] + 1;
        const int idle = occ > 0 ? 0 : p.ctl[1] + 1;
        const bool stop = *p.stop != 0;
        const bool go = !stop && it < p.max_iter && idle < p.idle_max;
        p.ctl[0] = go ? it : 0;
        p.ctl[1] = go ? idle : 0;
        p.ctl[3] = go ? 0 : (stop ? 1 : (it >= p.max_iter ? 2 : 3));
        cudaGraphSetConditional(p.cond, go ? 1u : 0u);
        unsigned sw = 0;
        while ((1 << sw) < ymax) ++sw;
        cudaGraphSetConditional(p.cond_step, ymax > 0 ? sw : (unsigned)p.nsizes);
        if (p.after_tick) cudaGraphSetConditional(p.cond_fin, p.fin[p.slots] > 0 ? 1u : 0u);
    }
}

// Residual blocks of the finishing slots: block b of every such slot, in the
// assignment k_residual uses for a grid of nblk blocks.
__global__ void k_loop_finish(const LoopParams p)
{
    const int nf = p.fin[p.slots];
    for (int f = 0; f < nf; ++f) {
        const int j = p.fin[f];
        float *dj = p.data + (size_t)j * p.ndata;
        residual_block(dj, p.dobs[j], dj, p.ndata, p.part + (size_t)j * p.nblk, blockIdx.x, p.nblk);
        __syncthreads();                       // the block's shared scratch is reused by the next slot
    }
}

// The finishing slots' misfits (one block of 1024 threads, the tree of
// k_reduce_phi), each published to the host after its value.
__global__ void k_loop_reduce(const LoopParams p)
{
    const int nf = p.fin[p.slots];
    for (int f = 0; f < nf; ++f) {
        const int j = p.fin[f];
        reduce_partials(p.part + (size_t)j * p.nblk, p.nblk, p.scale, p.phi[j]);
        if (threadIdx.x == 0) {
            __threadfence_system();
            p.done[j] = p.seen[j];
        }
        __syncthreads();
    }
}

// Posts request `seq` into slot `slot` with its data and misfit pointers; the
// writes of the work before it on the stream (the slot's model preparation and
// field zeroing) are complete, and the post is written last.
__global__ void k_loop_post(int *post, const float **dobs_tbl, double **phi_tbl, int slot, int seq,
                            const float *dobs, double *phi)
{
    dobs_tbl[slot] = dobs;
    phi_tbl[slot] = phi;
    __threadfence();
    *reinterpret_cast<volatile int *>(post + slot) = seq;
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

}  // namespace

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launch()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launches() { return t_launches; }

int launch_prep(const hv_handle *h, const float *m, const float *v, int k, float *C, float *b, cudaStream_t st)
{
    dim3 grid((h->NX + 127) / 128, h->NZ);
    k_prep<<<grid, 128, 0, st>>>(m, v, k, C, b, h->nz, h->nx, h->nb, h->NZ, h->NX, h->P, h->fsize, h->dt, h->h);
    return cuda_check("k_prep launch");
}

int launch_finalize(const hv_handle *h, const float *m, double *img, int fmt, int G, int k, float *out32,
                    double *out64, double *scratch, cudaStream_t st)
{
    dim3 gg((h->NX + 127) / 128, h->NZ, k), gx((h->nx + 127) / 128, h->NZ, k), gz((h->nx + 127) / 128, h->nz, k);
    k_fold_g<<<gg, 128, 0, st>>>(img, fmt, G, k, h->NZ, h->NX, h->P, h->fsize);
    HV_RT_INTERNAL(cuda_check("k_fold_g launch"));
    k_fold_x<<<gx, 128, 0, st>>>(img, h->nx, h->nb, h->NZ, h->NX, h->P, h->fsize, scratch);
    HV_RT_INTERNAL(cuda_check("k_fold_x launch"));
    k_fold_z<<<gz, 128, 0, st>>>(m, scratch, h->nz, h->nx, h->nb, h->NZ, h->h, out32, out64);
    return cuda_check("k_fold_z launch");
}

int launch_partial_image(const hv_handle *h, const float *m, const double *img, int fmt, int G, int k, double *out,
                         cudaStream_t st)
{
    dim3 grid((h->NX + 127) / 128, h->NZ, k);
    k_partial_image<<<grid, 128, 0, st>>>(m, img, fmt, G, k, h->nz, h->nx, h->nb, h->NZ, h->NX, h->P, h->fsize, h->h,
                                          out);
    return cuda_check("k_partial_image launch");
}

int launch_fold_ext(const hv_handle *h, const double *ext, int k, float *out32, double *out64, cudaStream_t st)
{
    dim3 grid((h->nx + 127) / 128, h->nz, k);
    k_fold_ext<<<grid, 128, 0, st>>>(ext, h->nz, h->nx, h->nb, h->NZ, h->NX, out32, out64);
    return cuda_check("k_fold_ext launch");
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

int launch_count_nonfinite(const float *x, size_t n, unsigned long long *count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (n == 0) return HV_OK;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 152 * 8);
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, st>>>(x, n, count);
    return cuda_check("k_count_nonfinite launch");
}

int launch_loop_control(const LoopParams &p, cudaStream_t st, bool pdl)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(1);
    lc.blockDim = dim3(256);
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&lc, k_loop_control, p);
    if (e != cudaSuccess) return hvi::fail(HV_ECUDA, "k_loop_control launch: %s", cudaGetErrorString(e));
    return cuda_check("k_loop_control launch");
}

int launch_loop_finish(const LoopParams &p, cudaStream_t st)
{
    k_loop_finish<<<p.nblk, 256, 0, st>>>(p);   // 256 threads and nblk blocks: the misfit's fixed tree
    HV_RT_INTERNAL(cuda_check("k_loop_finish launch"));
    k_loop_reduce<<<1, 1024, 0, st>>>(p);
    return cuda_check("k_loop_reduce launch");
}

int launch_loop_post(int *post, const float **dobs_tbl, double **phi_tbl, int slot, int seq, const float *dobs,
                     double *phi, cudaStream_t st)
{
    k_loop_post<<<1, 1, 0, st>>>(post, dobs_tbl, phi_tbl, slot, seq, dobs, phi);
    return cuda_check("k_loop_post launch");
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
