// hv_internal.h -- private declarations shared by the libhv translation units.
#pragma once

#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <complex>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hv.h"

#define HV_RT_INTERNAL(call)                                                                          \
    do {                                                                                              \
        int r_ = (call);                                                                              \
        if (r_ != HV_OK) return r_;                                                                   \
    } while (0)

#include <nvtx3/nvToolsExt.h>

namespace hvi {

// An NVTX range over one library call: profilers that record NVTX show the
// call's name over its launches; without one attached it costs a few
// nanoseconds (header-only NVTX, no link-time dependency).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};


// ---------------------------------------------------------------- status
int fail(int code, const char *fmt, ...);
inline int ok() { return HV_OK; }
// hv_linalg.cpp: eigenvalues (descending) and eigenvectors (columns, row-major) of a
// Hermitian n x n matrix; inverse of a small nonsingular matrix.
int hermitian_eig(int n, std::vector<std::complex<double>> A, std::vector<double> &w,
                  std::vector<std::complex<double>> &V);
int small_inverse(int n, std::vector<std::complex<double>> M, std::vector<std::complex<double>> &inv);
int approx_device(const hv_approx *a);   // device a Hessian approximation lives on

// ---------------------------------------------------------------- schedule
enum { ACT_FORWARD = 0, ACT_SAVE = 1, ACT_RESTORE = 2, ACT_ADVANCE = 3, ACT_ADJOINT = 4 };
struct Action {
    int op, a0, a1;
};
long long seg_cost(long long L, int f);
int build_schedule(int nt, int slots, std::vector<Action> &out, long long *n_advances);

// ---------------------------------------------------------------- geometry
// Fields live on the padded grid (NZ x NX) inside a ghost band of GH = 4 zero
// cells on every side: padded node (z, x) sits at offset (z + 4) * P + (x + 4)
// of a field of `rows` = NZ + 8 rows and pitch P (a multiple of 4 floats, so
// every row and every 4-aligned column starts on a 16-byte boundary).  The
// ghost band is never written, which gives the Dirichlet zeros of the
// stencil without bounds checks.
constexpr int GH = 4;

// Tiling of one kernel configuration: TX x TZ interior points per CTA.
struct Tiling {
    int TX, TZ, ntx, ntz, ntiles;
};

// Receivers of every shot grouped by tile (for fused sampling/injection).
struct RecTiles {
    int TX = 0, TZ = 0, ntiles = 0;
    int *off = nullptr;   // [ns][ntiles+1] start of each tile's receivers
    int *rec = nullptr;   // [ns][nr] receiver index, tile-sorted
    int *pos = nullptr;   // [ns][nr] field offset of that receiver
};

}  // namespace hvi

struct hv_handle {
    unsigned long long serial = 0;   // unique per hv_create in the process (a later handle may reuse the address)
    int device = 0;
    int nz = 0, nx = 0, nb = 0, NZ = 0, NX = 0;
    int P = 0, rows = 0;
    size_t fsize = 0;            // floats per field (rows * P rounded up to 64)
    double h = 0, dt = 0, f0 = 0, t0 = 0, vmax = 0, R = 0, sigma = 1;
    int ns = 0, nr = 0, nt = 0;
    // device arrays owned by the handle
    float *wavelet = nullptr;    // [nt]   s(n dt)
    float *az = nullptr;         // [NZ]   sponge a = q dt / 2 along z
    float *ax = nullptr;         // [NX]   sponge a = q dt / 2 along x
    int *src_zx = nullptr;       // [ns][2] padded (z, x) of each source
    int *rec_zx = nullptr;       // [ns*nr][2] padded (z, x) of each receiver
    int *status = nullptr;       // device status word (HV_ETIMEOUT if a bounded wait ran out)
    unsigned long long wait_ns = 2000000000ull;   // limit of every device wait (hv_set_wait_limit)
    bool inject_wait = false;    // next dataflow-ordered step waits for a count nothing reaches (hv_inject_wait_timeout)
    std::vector<int> h_src_zx, h_rec_zx;
    std::mutex mu;
    std::map<long long, hvi::RecTiles> rectiles;                 // keyed by TX * 65536 + TZ
    std::map<int, std::vector<hvi::Action>> schedules;           // keyed by slots
    // tile configuration per kernel kind (HV_K_FWD, HV_K_ADVANCE, HV_K_ADJ); see hv_autotune
    int cfg[3] = {0, 0, 0};
    // CUDA graphs of the H v launch sequence (hv_set_graphs), keyed by workspace and shape
    bool graphs_on = false;
    cudaStream_t capture_stream = nullptr;
    // how stencil steps are ordered after one another (hv_set_launch_mode)
    int launch_mode = HV_LAUNCH_PDL;
    // recomputation runs two steps per launch where it can (hv_set_step_fusion)
    bool fuse_steps = false;
    // H v with every level stored on the shared-memory-resident kernels (hv_set_resident)
    bool resident = false;
    // high-pass filter of the PSF and PDO builds (hv_set_highpass): cutoff rho_c [rad/m], 0 = off
    double highpass = 0.0;
    // imaging accumulation (hv_set_image_precision): false = per-step FP32 sums over
    // a shot group added to double-float images; true = every shot's product added in FP64
    bool img_f64 = false;
    std::map<std::string, cudaGraphExec_t> graphs;
    std::deque<std::string> graph_order;   // keys, oldest first (the cache holds at most kMaxGraphs)
    // profiling (hv_profile)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_rec;
};

namespace hvk {

// Tile configurations (hv_stencil.cu): the menu size and the tiling of one entry.
int tile_menu_size();
int max_tiles(const hv_handle *h);    // most tiles any menu entry cuts the handle's grid into
void menu_info(int cfg, int *info);   // {TX, TZ, threads, stages, shot groups per CTA}
hvi::Tiling tiling(const hv_handle *h, int cfg);
int prepare_kernels(const hv_handle *h);
int adj_f64_cfg();   // tile configuration of the FP64-image adjoint (hv_set_image_precision)

// Tensor maps of one call's workspace, viewed as an array of fields
// (x, z, field index): `halo` copies a tile with its 4-cell halo, `pt` the
// tile's own points.  Opaque CUtensorMap bytes (128 each).
constexpr int kMaxTileMenu = 16;
struct TmaMaps {
    alignas(64) unsigned char halo[kMaxTileMenu][128];   // per tile configuration
    alignas(64) unsigned char pt[kMaxTileMenu][128];
    alignas(64) unsigned char halo8[kMaxTileMenu][128];  // 8-cell halo (two fused steps)
    void *ws = nullptr;
    long long nfields = 0;
};
int make_maps(const hv_handle *h, void *ws, long long nfields, TmaMaps *m);

// Ordering of a stencil step after the previous ones (see hv_set_launch_mode).
// cnt: per (shot group, tile) counts of completed step items in this call, or
// nullptr; a step adds one per (vector, group, tile) it finishes.  With
// `flow`, a CTA waits only until its tile and the 8 neighbours have reached
// `need` (the items of all earlier steps of the call) instead of waiting for
// the whole previous grid; the caller sets it only when the previous kernel on
// the stream was a counting stencil step with the same tiling.
struct StepDeps {
    int *cnt = nullptr;
    int need = 0;
    bool flow = false;
};

struct FwdLaunch {
    const float *u_cur, *u_prev;   // field batches [ns][fsize]
    float *u_next;                 // may be nullptr (Born-only groups never write u)
    const float *C;                // [fsize] m^2 dt^2 / h^2
    const float *b;                // [k][fsize] 2 dm / m (Born) or nullptr
    const float *du_cur;           // [k][ns][fsize] Born field at n
    float *du_io;                  // [k][ns][fsize] Born field at n-1 in, n+1 out
    float *d_u;                    // [ns][nt][nr] samples of u^{n+1} or nullptr
    float *d_du;                   // [k][ns][nt][nr] samples of du^{n+1} or nullptr
    int n, k;
    // Without Born fields: models advanced in one launch (0 or 1: one).  Model
    // i has coefficient field C + i fields, field batches starting `i ns`
    // fields after u_cur, u_prev and u_next, and data d_u + i ns nt nr.
    int models;
    // Without Born fields: per-model step counters (device, [models]; see k_fwd),
    // or nullptr.  With them, n counts launches and u_cur is the first field of
    // the models' rings (model i: 3 ns fields from u_cur + 3 ns i fields).
    const int *slot_join;
    bool plain;                    // launch without programmatic dependent launch whatever the handle's mode
    StepDeps deps;
};
int launch_fwd(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const FwdLaunch &a,
               cudaStream_t st);

// Two fused forward steps without Born fields or receivers (hv_stencil.cu, k_fwd2).
struct Fwd2Launch {
    const float *u_cur, *u_prev;   // u^n, u^{n-1}
    float *u_next1, *u_next2;      // u^{n+1}, u^{n+2} (distinct from the inputs)
    const float *C;
    int n;                         // first step; n + 1 < nt
};
int launch_fwd2(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const Fwd2Launch &a,
                cudaStream_t st);

struct AdjLaunch {
    const float *u;                // u^n field batch [ns][fsize]
    const float *lam1;             // [k][ns][fsize] lam^{n+1}
    float *lam_io;                 // [k][ns][fsize] lam^{n+2} in, lam^n out
    const float *C;
    const float *r;                // adjoint source data, [k or 1][ns][nt][nr]
    int r_per_vector;              // 1 if r has a vector dimension
    float rscale;                  // multiplies r (h^2 / sigma^2 or h^2)
    double *img;                   // [G][k][fsize] partial images, double-float (hi, lo) FP32 pairs (or FP64)
    bool img_f64;                  // every shot's product added in FP64 (hv_set_image_precision)
    int n, k, G;
    StepDeps deps;
};
int launch_adj(const hv_handle *h, int cfg, const hvi::RecTiles &rt, const TmaMaps &maps, const AdjLaunch &a,
               cudaStream_t st);
int adj_groups(const hv_handle *h);
// CTAs of one model in a forward step (no Born fields) with tile configuration cfg.
int fwd_ctas_per_model(const hv_handle *h, int cfg);

// Shared-memory-resident H v kernels (every forward level stored, grids whose
// padded field fits twice in a CTA's shared memory): which = 0 the forward
// fields of all shots (writes Q^n = Lh u^n + s_n into the history), 1 the Born
// fields of all (shot, vector) pairs (writes the Born data), 2 the adjoint
// fields and per-pair images.
struct ResLaunch {
    void *base;                    // workspace base (field 0)
    const float *C, *b;            // C, b [k]
    float *q;                      // Q history: nt batches of ns fields
    float *dd;                     // Born data [k][ns][nt][nr]
    float rscale;                  // adjoint source scale
    void *img;                     // per-pair images [ns][k][fsize] double-float pairs
    const int *rec, *pos;          // receivers of each shot ([ns][nr], any order)
    int k;
};
bool resident_fits(const hv_handle *h);
int launch_resident(const hv_handle *h, int which, const ResLaunch &a, cudaStream_t st);

int launch_prep(const hv_handle *h, const float *m, const float *v, int k, float *C, float *b, cudaStream_t st);

// PSF approximation (hv_psf.cu): lattice of sample points and its batches.
struct PsfGeo {
    int nz, nx;       // interior grid
    int S, B, R;      // lattice spacing, batches per axis, window radius (B S - 1) / 2
    int na, nb;       // sample points along z and x
    int cz0, cx0;     // first sample point
    int k = 0, vpc = 1;   // apply launches: vectors, vectors per CTA
};
// Low-rank-symbol PsiDO and PDO probing (hv_pdo.cu).
constexpr int kLrMaxTerms = 32;
struct LrGeo {
    int nz = 0, nx = 0, r = 0;   // grid, terms (sample frequencies)
    double h = 0, win = 0;       // spacing; separation window radius rho0 sin(pi / r) [rad/m]
    int iz[kLrMaxTerms] = {}, ix[kLrMaxTerms] = {};   // signed DFT indices of the snapped samples
    float rho[kLrMaxTerms] = {};                      // their radii [rad/m]
};
struct LrSym {
    LrGeo g;
    float2 *a = nullptr;   // [r][nz][nx] symbol factors a_k(x)
    float2 *b = nullptr;   // [r][nz][nx] symbol factors b_k(xi), DFT order
    float2 *Y = nullptr, *V = nullptr;   // scratch: r x kb spectra, kb spectra
    float *T = nullptr;                  // scratch: kb real fields (B^T v of B B^T v)
    bool spd = false;                    // square-root symbol: the approximation is B B^T
    int kb = 1;                          // vectors per apply batch
    cufftHandle pf = 0, pi = 0;          // build: one forward, r inverse (C2C, nz x nx)
    cufftHandle pfb = 0, pib = 0;        // apply: kb forward, r x kb inverse (pib: not with fused transforms)
    bool pf_ok = false, pi_ok = false, pfb_ok = false, pib_ok = false;
    bool fused = false;                  // applies through the fused transforms of hv_lrfft.cu
    float2 *tw = nullptr;                // their twiddle tables: nz, then nx entries
    void *part = nullptr;                // their partial sums over term chunks (more than 8 terms)
    cudaEvent_t done = nullptr;          // last use of the scratch
    std::mutex *mu = nullptr;
};
int lr_samples(int nz, int nx, double h, double rho0, int r, LrGeo &g);
int lr_create(LrSym &L, const LrGeo &g);
void lr_destroy(LrSym &L);
int launch_pdo_probe(const LrGeo &g, float *v, cudaStream_t st);
int pdo_columns(LrSym &L, const float *Hvp, cudaStream_t st);
constexpr int kLrForward = 0, kLrTranspose = 1, kLrGram = 2;   // B v, B^T v, B B^T v
int lr_apply(LrSym &L, const float *v, int k, float *out, cudaStream_t st, int op = kLrForward);
int pdo_sqrt(const LrSym &src, LrSym &out, cudaStream_t st);
// The fused transforms of the low-rank-symbol applies (hv_lrfft.cu): power-of-two
// grids with 16 <= nz, nx <= 512.  forward: out = Re sum_k a_k F^-1 (b_k V) from
// the spectra V of nq vectors; transpose: V = (1/N) sum_k conj(b_k) F (conj(a_k) w).
bool lr_fused_default();
bool lr_fused_supported(int nz, int nx);
int lr_fused_init(LrSym &L);
int lr_fused_forward(const LrSym &L, const float2 *V, int nq, float *out, cudaStream_t st);
int lr_fused_transpose(const LrSym &L, const float *w, int nq, float2 *V, cudaStream_t st);
void launch_sqrt_real(const float2 *in, float2 *out, size_t n, cudaStream_t st);
// The high-pass filter of the approximations (hv_highpass.cu): F_hp v =
// Re F^-1 (phi(|xi|) F v), phi(rho) = 1 - exp(-rho^2 / (2 rho_c^2)).
struct Highpass {
    int nz = 0, nx = 0, kmax = 0;
    double h = 0, rho_c = 0;
    float *tab = nullptr;        // [nz][nx/2+1] phi / (nz nx)
    float2 *spec = nullptr;      // [kmax][nz][nx/2+1]
    cufftHandle fwd = 0, inv = 0, fwd1 = 0, inv1 = 0;   // R2C / C2R, batch kmax and batch 1
    bool fwd_ok = false, inv_ok = false, fwd1_ok = false, inv1_ok = false;
};
int highpass_create(Highpass &F, int nz, int nx, double h, double rho_c, int kmax);
void highpass_destroy(Highpass &F);
int highpass_apply(Highpass &F, const float *v, int k, float *out, cudaStream_t st);   // out may be v
// A^-1 of the Matern prior by the 2D DCT (hv_dct.cu): one real 2D DFT of the
// reordered field, a kernel that forms the DCT coefficients, divides by the
// eigenvalues and rebuilds the half spectrum, and the inverse DFT.
struct Dct2 {
    int n1 = 0, n2 = 0, kmax = 0;   // transform grid (a one-column field is taken as 1 x nz)
    float2 *tw = nullptr;           // (cos, sin)(pi a / (2 n1)), a <= n1, then the same for n2
    float *inv = nullptr;           // [nz][nx] 1 / (lambda nz nx)
    float *w = nullptr;             // [kmax][nz][nx] reordered fields
    float2 *s1 = nullptr, *s2 = nullptr;   // [kmax][n1][n2/2+1] half spectra
    cufftHandle f = 0, i = 0, f1 = 0, i1 = 0;
    bool f_ok = false, i_ok = false, f1_ok = false, i1_ok = false;
};
int dct_create(Dct2 &D, int nz, int nx, double h, double delta, double gamma, int kmax);
void dct_destroy(Dct2 &D);
int dct_apply(Dct2 &D, const float *v, int k, float *out, cudaStream_t st);   // out = A^-1 v, out may be v
// Matern prior and the low-rank approximation (hv_lowrank.cu).
struct Prior {
    int nz = 0, nx = 0;
    double h = 0, delta = 0, gamma = 0;
    float *Cz = nullptr, *Cx = nullptr;   // orthonormal DCT-II matrices
    float *inv = nullptr;                 // 1 / (delta + gamma lambda_kl) in DCT order
    double *Czd = nullptr, *Cxd = nullptr, *invd = nullptr;   // the same in FP64 (low-rank build)
    Dct2 dct;                             // A^-1 in FP32 (fields in batches of up to dct.kmax)
    float *tmp = nullptr;                 // scratch, 2 tmp_k fields
    double *tmpd = nullptr;
    int tmp_k = 0, tmpd_k = 0;
    cublasHandle_t blas = nullptr;
    bool blas_ok = false;
};
int prior_create(Prior &P, int nz, int nx, double h, double delta, double gamma);
void prior_destroy(Prior &P);
int prior_reserve(Prior &P, int k);   // scratch for applies of up to k fields (allocated here, not later)
int prior_A(const Prior &P, const float *v, float *out, int k, cudaStream_t st);
int prior_Ainv(Prior &P, const float *v, float *out, int k, cudaStream_t st);
int prior_R(Prior &P, const float *v, float *out, int k, cudaStream_t st);
int prior_Rinv(Prior &P, const float *v, float *out, int k, cudaStream_t st);
struct LowRank {
    Prior prior;
    int r = 0;
    size_t N = 0;
    std::vector<double> lam;   // eigenvalues, descending
    float *V = nullptr;        // [r][N], V^T R V = I
    float *W = nullptr;        // [r][N], W = A V
    float *U = nullptr;        // [r][N], U = A W = R V
    double *w = nullptr;       // [2r]: Lambda, then S_r = 1 - (Lambda + 1)^-1/2
    double *c = nullptr;       // [xk][r] scratch coefficients
    float *x = nullptr;        // [xk][N] scratch fields
    double *red = nullptr;     // reduction partials for xk vectors
    int xk = 0;                // vectors the scratch holds
    cudaEvent_t done = nullptr;   // last use of the scratch
    std::mutex *mu = nullptr;     // applies from several streams run one after another
};
// Y_in = H_d Omega [k][N]; `hessian(X, kk, out)` applies H_d to kk fields.
int build_lowrank(LowRank &L, const float *Y_in, int k, int rank, size_t N,
                  const std::function<int(const float *, int, float *)> &hessian, cudaStream_t st);
void lowrank_destroy(LowRank &L);
int lowrank_apply(LowRank &L, const float *v, int k, float *out, int mode, cudaStream_t st);

// PSF+ (hv_psfplus.cu): the low-rank symbol refined from PSF rows and PDO columns.
int build_psfplus(const PsfGeo &pg, const float *psf, const LrSym &pdo, double tol, bool spd, LrSym &out,
                  cudaStream_t st);

int launch_psf_impulses(const PsfGeo &g, float *v, cudaStream_t st);   // v zeroed, [B*B][nz][nx]
int launch_psf_extract(const PsfGeo &g, const float *Hv, float *psf, cudaStream_t st);
int launch_psf_apply(const PsfGeo &g, const float *psf, const float *v, int k, float *out, cudaStream_t st);
int psf_apply_smem_bytes(int S, int R, int nvec);   // dynamic shared memory of the apply kernel
// Image formats (img_at): 0 double-float pairs per shot group, 1 FP64
// per shot group (both in the field layout), 2 one dense FP64 [k][NZ][NX] image.
constexpr int kImgPairs = 0, kImgF64 = 1, kImgDense = 2;
// The fold of the group images onto the interior; the group sums overwrite
// group 0's image; scratch: k NZ nx doubles apart from img (the call's Born /
// adjoint field region, free by then).
int launch_finalize(const hv_handle *h, const float *m, double *img, int fmt, int G, int k, float *out32,
                    double *out64, double *scratch, cudaStream_t st);
int launch_partial_image(const hv_handle *h, const float *m, const double *img, int fmt, int G, int k, double *out,
                         cudaStream_t st);
int launch_fold_ext(const hv_handle *h, const double *ext, int k, float *out32, double *out64, cudaStream_t st);
int launch_residual(const hv_handle *h, const float *d, const float *dobs, float *r, double *partials,
                    int nblocks, cudaStream_t st);
int launch_reduce_phi(const double *partials, int nblocks, double scale, double *phi, cudaStream_t st);

// The device-resident misfit loop (hv_engine_serve and the kernels of its
// graph body, hv_kernels.cu).  One iteration is one body of a switch: the
// forward step of the occupied slots launched over the first 1, 2, 4, ...
// slots (the smallest prefix covering the highest occupied one), then
// k_loop_control (admission, steps, conditions), then, if any slot took its
// last step, k_loop_finish and k_loop_reduce form those misfits; or, with no
// slot occupied (and first in every launch), k_loop_control alone.
constexpr int kLoopFreeSlot = 1 << 30;    // a slot_join entry that makes k_fwd skip the slot
struct LoopParams {
    int slots, nt, nblk;
    size_t ndata;                  // data floats per slot (ns nt nr)
    double scale;                  // 1 / (2 sigma^2)
    int max_iter, idle_max;        // bounds of one launch of the loop
    int *post;                     // [slots] sequence number of the last request posted into the slot
    int *seen;                     // [slots] sequence number of the last request admitted
    int *step;                     // [slots] step the slot takes in this iteration (-1: free)
    int *join;                     // [slots] k_fwd's slot_join table: -step, or kLoopFreeSlot
    int *fin;                      // [slots + 1] the slots taking their last step in this iteration, count last
    int *ctl;                      // [4] iteration, idle iterations, occupied slots, exit reason
    const float *const *dobs;      // [slots] observed data of each slot's request
    double *const *phi;            // [slots] where each slot's misfit goes
    float *data;                   // [slots][ndata]
    double *part;                  // [slots][nblk]
    volatile int *ack;             // [slots] host-mapped: sequence number admitted
    volatile int *done;            // [slots] host-mapped: sequence number whose misfit is written
    volatile int *stop;            // host-mapped: nonzero ends the loop at the end of the iteration
    cudaGraphConditionalHandle cond, cond_step, cond_fin;   // while; switch over step launches; if a misfit finishes
    int nsizes;                    // step launches of the switch; body nsizes has no step
    int after_tick;                // k_loop_control runs behind a step (advance the slots, list the finishing ones)
};
int launch_loop_control(const LoopParams &p, cudaStream_t st, bool pdl);
int launch_count_nonfinite(const float *x, size_t n, unsigned long long *count, cudaStream_t st);
int launch_loop_finish(const LoopParams &p, cudaStream_t st);
int launch_loop_post(int *post, const float **dobs_tbl, double **phi_tbl, int slot, int seq, const float *dobs,
                     double *phi, cudaStream_t st);
int launch_copy_wavefield(const hv_handle *h, const float *u, float *out, cudaStream_t st);
int launch_zero_ghosts(const hv_handle *h, float *f, long long nfields, cudaStream_t st);
int launch_setup(hv_handle *h, cudaStream_t st);

// Skinny dense products over grid fields (hv_blas.cu); deterministic chunked
// reductions (rows_dot: FP64; coef: FP32 inside a chunk, FP64 across chunks).
// scratch: the FP64 partials, rows_dot_scratch / coef_scratch doubles.
int chunks_of(size_t N);
size_t rows_dot_scratch(int k, size_t N);
size_t coef_scratch(int r, int k, size_t N);
// out[q] = scale sum_e A[q][e] B[q][e], q < k
int rows_dot(const float *A, const float *B, double *out, int k, size_t N, double scale, double *scratch,
             cudaStream_t st);
// C[q][j] = w[j] sum_e M[j][e] X[q][e] (w may be null: 1), j < r, q < k
int coef(const float *M, int r, const float *X, int k, size_t N, const double *w, double *C, double *scratch,
         cudaStream_t st);
// out[q][e] = base[q][e] + sign sum_j C[q][j] M[j][e] (base may be null: 0; out may be base), r <= 256
int combine(const float *M, int r, const double *C, int k, size_t N, const float *base, float sign, float *out,
            cudaStream_t st);

// Process-wide kernel launch counter (hv_kernel_launches).
void count_launch();
long long launches_so_far();
long long thread_launches();   // kernels launched by the calling thread

}  // namespace hvk

// A built Hessian approximation (hv_approx_*).
struct hv_approx {
    int kind = 0;           // 0: PSF, 1: PDO, 2: PSF+ (1 and 2: low-rank symbol), 3: LR
    int device = -1;
    hvk::PsfGeo g{};
    float *psf = nullptr;   // [na * nb][2R+1][2R+1]
    hvk::LrSym lr;          // PDO / PSF+: symbol factors, weights, FFT plans
    hvk::LowRank low;       // LR: prior and generalised eigenpairs
    int nz = 0, nx = 0;
};
