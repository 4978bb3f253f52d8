/*
 * hv_oracle.c -- plain FP64 CPU oracle for the matrix-free Gauss-Newton
 * Hessian-vector product of 2D acoustic seismic inversion
 * (Hu, Alger, Nammour, Ghattas: "Accelerating seismic inversion and
 * uncertainty quantification with efficient high-rank Hessian
 * approximations", arXiv 2507.10804).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and it is deliberately slow: every
 * operator is written out as its plain definition, one loop per operator,
 * with no fusion, blocking or reordering.  Compiled with -O2
 * -ffp-contract=off so that x86 and Arm hosts round identically.
 *
 * What it computes (paper section 2, eq. (pde), eq. (data), eq. (grad), and
 * section 3, "two wave equations per source"):
 *
 *   H_d v = E^T G^T S^{-T} P^T Gamma^{-1} P S^{-1} G E v
 *
 * for the discrete wave operator described below.  The paper fixes only the
 * continuous equation (1/m^2) u_tt - lap(u) = s(t) delta(x - x_s) with m the
 * wave speed; the discretisation follows the readings listed in the design
 * notes: 2nd order in time, 8th order in space, an absorbing sponge on all
 * four sides, Ricker source, point receivers.
 *
 * Discrete operator (padded grid NZ = nz + 2 nb rows, NX = nx + 2 nb columns,
 * row-major with x fastest, zero values outside the padded grid):
 *
 *   L u       = (1/h^2) sum_{k=-4..4} c_|k| (u[z][x+k] + u[z+k][x]),
 *               c0 = -205/72, c1 = 8/5, c2 = -1/5, c3 = 8/315, c4 = -1/560
 *   sponge    : (1/m^2)(u_tt + q u_t) - L u = f with a damping RATE q [1/s]
 *               that is zero in the interior (where the equation is exactly
 *               eq. (pde)) and does not depend on m:
 *               q = max(q_z, q_x), q_a(d) = q_max (d/(nb h))^2, d the distance
 *               into the sponge (h for the first sponge cell),
 *               q_max = 3 vmax ln(1/R) / (2 nb h)
 *   rows n=0..nt-1 of S U = F (T is the damped second time difference):
 *               (1/m^2) (T u)^n - L u^n = f^n,  u^0 = u^{-1} = 0,
 *               (T u)^n = (u^{n+1} - 2u^n + u^{n-1})/dt^2 + q (u^{n+1} - u^{n-1})/(2 dt)
 *               i.e. M2 u^{n+1} - K u^n + M0 u^{n-1} = f^n with
 *               M2 = (1/m^2)(1/dt^2 + q/(2 dt)), M0 = (1/m^2)(1/dt^2 - q/(2 dt)),
 *               K  = 2/(m^2 dt^2) + L
 *   source    : f^n = s(n dt)/h^2 at the shot node (1/h^2 = discrete delta),
 *               s(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)
 *   receivers : P: d[n][r] = u^{n+1}[rec_r]
 *   Born      : S dU = G dm, (G dm)^n = (2 dm/m^3) (T u)^n  (S depends on m
 *               only through the factor 1/m^2)
 *   adjoint   : S^T lam = g:  M2 lam^n = K lam^{n+1} - M0 lam^{n+2} + g^n,
 *               lam^{nt} = lam^{nt+1} = 0
 *   imaging   : G^T lam = sum_n (2/m^3) lam^n (T u)^n
 *   noise     : Gamma_noise = sigma^2 I (paper section 2.1)
 *   extension : E copies the interior model into the sponge by edge
 *               replication; E^T sums sponge entries onto the edge cells.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* Problem description; mirrored field by field by oracle/oracle.py. */
typedef struct {
    int nz, nx, nb;         /* interior rows, interior columns, sponge width  */
    double h;               /* grid spacing [m]                               */
    int nt;                 /* number of time steps                           */
    double dt;              /* time step [s]                                  */
    double f0, t0;          /* Ricker peak frequency [Hz] and delay [s]       */
    double vmax;            /* velocity that sizes the sponge [m/s]           */
    double R;               /* sponge target reflection coefficient           */
    double sigma;           /* noise standard deviation                       */
    int ns, nr;             /* shots, receivers per shot                      */
    const int *src_iz, *src_ix;   /* [ns]    interior node of each shot        */
    const int *rec_iz, *rec_ix;   /* [ns*nr] interior node of each receiver    */
} or_problem;

static const double OR_C[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

static int NZ_(const or_problem *P) { return P->nz + 2 * P->nb; }
static int NX_(const or_problem *P) { return P->nx + 2 * P->nb; }

int or_version(void) { return 1; }

/* ------------------------------------------------------------------------ */
/* Source wavelet: Ricker, s(t) = (1 - 2 a) exp(-a), a = pi^2 f0^2 (t - t0)^2 */
void or_ricker(int nt, double dt, double f0, double t0, double *s)
{
    for (int n = 0; n < nt; ++n) {
        double tau = n * dt - t0;
        double a = M_PI * M_PI * f0 * f0 * tau * tau;
        s[n] = (1.0 - 2.0 * a) * exp(-a);
    }
}

/* Sponge damping rate q [1/s] on the padded grid (zero in the interior). */
void or_sponge_q(const or_problem *P, double *q)
{
    int NZ = NZ_(P), NX = NX_(P), nb = P->nb;
    double L = nb * P->h;
    double q_max = (nb > 0) ? 3.0 * P->vmax * log(1.0 / P->R) / (2.0 * L) : 0.0;
    for (int z = 0; z < NZ; ++z) {
        double dz = 0.0;
        if (z < nb) dz = (nb - z) * P->h;
        else if (z >= nb + P->nz) dz = (z - (nb + P->nz) + 1) * P->h;
        for (int x = 0; x < NX; ++x) {
            double dx = 0.0;
            if (x < nb) dx = (nb - x) * P->h;
            else if (x >= nb + P->nx) dx = (x - (nb + P->nx) + 1) * P->h;
            double qz = q_max * (dz / L) * (dz / L);
            double qx = q_max * (dx / L) * (dx / L);
            q[(size_t)z * NX + x] = (nb > 0) ? (qz > qx ? qz : qx) : 0.0;
        }
    }
}

/* E: edge-replicating extension of an interior field to the padded grid. */
void or_extend(const or_problem *P, const double *m, double *mext)
{
    int NZ = NZ_(P), NX = NX_(P), nb = P->nb;
    for (int z = 0; z < NZ; ++z) {
        int iz = z - nb;
        if (iz < 0) iz = 0;
        if (iz > P->nz - 1) iz = P->nz - 1;
        for (int x = 0; x < NX; ++x) {
            int ix = x - nb;
            if (ix < 0) ix = 0;
            if (ix > P->nx - 1) ix = P->nx - 1;
            mext[(size_t)z * NX + x] = m[(size_t)iz * P->nx + ix];
        }
    }
}

/* E^T: the exact transpose of or_extend (sum over each interior cell's copies). */
void or_fold(const or_problem *P, const double *gext, double *g)
{
    int NZ = NZ_(P), NX = NX_(P), nb = P->nb;
    memset(g, 0, sizeof(double) * (size_t)P->nz * P->nx);
    for (int z = 0; z < NZ; ++z) {
        int iz = z - nb;
        if (iz < 0) iz = 0;
        if (iz > P->nz - 1) iz = P->nz - 1;
        for (int x = 0; x < NX; ++x) {
            int ix = x - nb;
            if (ix < 0) ix = 0;
            if (ix > P->nx - 1) ix = P->nx - 1;
            g[(size_t)iz * P->nx + ix] += gext[(size_t)z * NX + x];
        }
    }
}

/* L u on the padded grid, zero outside (homogeneous Dirichlet ghosts). */
void or_laplacian(const or_problem *P, const double *u, double *Lu)
{
    int NZ = NZ_(P), NX = NX_(P);
    double ih2 = 1.0 / (P->h * P->h);
    for (int z = 0; z < NZ; ++z)
        for (int x = 0; x < NX; ++x) {
            double acc = 2.0 * OR_C[0] * u[(size_t)z * NX + x];
            for (int k = 1; k <= 4; ++k) {
                double ux = 0.0, uz = 0.0;
                if (x - k >= 0) ux += u[(size_t)z * NX + x - k];
                if (x + k < NX) ux += u[(size_t)z * NX + x + k];
                if (z - k >= 0) uz += u[(size_t)(z - k) * NX + x];
                if (z + k < NZ) uz += u[(size_t)(z + k) * NX + x];
                acc += OR_C[k] * (ux + uz);
            }
            Lu[(size_t)z * NX + x] = acc * ih2;
        }
}

/* Per-node coefficients of the time-stepping rows. */
typedef struct {
    const or_problem *P;
    size_t N;
    double *M2, *M0, *A;   /* A = 1/(m^2 dt^2), the diagonal part of K */
    double *m;             /* extended model                           */
    double *q;             /* sponge damping rate                      */
    double *Lbuf;          /* scratch for L w                          */
} or_ops;

static int ops_init(or_ops *O, const or_problem *P, const double *mext)
{
    O->P = P;
    O->N = (size_t)NZ_(P) * NX_(P);
    O->M2 = malloc(sizeof(double) * O->N);
    O->M0 = malloc(sizeof(double) * O->N);
    O->A = malloc(sizeof(double) * O->N);
    O->m = malloc(sizeof(double) * O->N);
    O->Lbuf = malloc(sizeof(double) * O->N);
    O->q = malloc(sizeof(double) * O->N);
    if (!O->M2 || !O->M0 || !O->A || !O->m || !O->Lbuf || !O->q) return -1;
    or_sponge_q(P, O->q);
    for (size_t p = 0; p < O->N; ++p) {
        double mm = mext[p];
        O->m[p] = mm;
        O->A[p] = 1.0 / (mm * mm * P->dt * P->dt);
        O->M2[p] = (1.0 / (mm * mm)) * (1.0 / (P->dt * P->dt) + O->q[p] / (2.0 * P->dt));
        O->M0[p] = (1.0 / (mm * mm)) * (1.0 / (P->dt * P->dt) - O->q[p] / (2.0 * P->dt));
    }
    return 0;
}

static void ops_free(or_ops *O)
{
    free(O->M2); free(O->M0); free(O->A); free(O->m); free(O->Lbuf); free(O->q);
}

/* One row of the recurrence: M2 next = K cur - M0 prev + src. */
static void row_solve(or_ops *O, const double *cur, const double *prev, const double *src, double *next)
{
    or_laplacian(O->P, cur, O->Lbuf);
    for (size_t p = 0; p < O->N; ++p) {
        double Kcur = 2.0 * O->A[p] * cur[p] + O->Lbuf[p];
        double pv = prev ? prev[p] : 0.0;
        next[p] = (Kcur - O->M0[p] * pv + src[p]) / O->M2[p];
    }
}

/* U = S^{-1} F.  F[n] (n = 0..nt-1) are the row right-hand sides; U[n] = u^{n+1}. */
static void solve_S(or_ops *O, const double *F, double *U)
{
    int nt = O->P->nt;
    size_t N = O->N;
    double *zero = calloc(N, sizeof(double));
    for (int n = 0; n < nt; ++n) {
        const double *cur = (n >= 1) ? U + (size_t)(n - 1) * N : zero;   /* u^n     */
        const double *prev = (n >= 2) ? U + (size_t)(n - 2) * N : zero;  /* u^{n-1} */
        row_solve(O, cur, prev, F + (size_t)n * N, U + (size_t)n * N);
    }
    free(zero);
}

/* Lam = S^{-T} G.  G[n] lives in unknown space (pairs with u^{n+1}); Lam[n] = lam^n. */
static void solve_ST(or_ops *O, const double *G, double *Lam)
{
    int nt = O->P->nt;
    size_t N = O->N;
    double *zero = calloc(N, sizeof(double));
    for (int n = nt - 1; n >= 0; --n) {
        const double *cur = (n + 1 <= nt - 1) ? Lam + (size_t)(n + 1) * N : zero;
        const double *prev = (n + 2 <= nt - 1) ? Lam + (size_t)(n + 2) * N : zero;
        row_solve(O, cur, prev, G + (size_t)n * N, Lam + (size_t)n * N);
    }
    free(zero);
}

/* Damped second time difference of the state,
 * D[n] = (T u)^n = (u^{n+1} - 2u^n + u^{n-1})/dt^2 + q (u^{n+1} - u^{n-1})/(2 dt). */
static void time_operator(const or_ops *O, const double *U, double *D)
{
    size_t N = O->N;
    int nt = O->P->nt;
    double dt = O->P->dt;
    for (int n = 0; n < nt; ++n)
        for (size_t p = 0; p < N; ++p) {
            double up1 = U[(size_t)n * N + p];
            double u0 = (n >= 1) ? U[(size_t)(n - 1) * N + p] : 0.0;
            double um1 = (n >= 2) ? U[(size_t)(n - 2) * N + p] : 0.0;
            D[(size_t)n * N + p] = (up1 - 2.0 * u0 + um1) / (dt * dt) + O->q[p] * (up1 - um1) / (2.0 * dt);
        }
}

static size_t src_node(const or_problem *P, int s)
{
    return (size_t)(P->src_iz[s] + P->nb) * NX_(P) + (P->src_ix[s] + P->nb);
}

static size_t rec_node(const or_problem *P, int s, int r)
{
    size_t i = (size_t)s * P->nr + r;
    return (size_t)(P->rec_iz[i] + P->nb) * NX_(P) + (P->rec_ix[i] + P->nb);
}

/* Forward wavefield of one shot: U[n] = u^{n+1}, n = 0..nt-1. */
static void shot_forward(or_ops *O, int s, double *U)
{
    const or_problem *P = O->P;
    size_t N = O->N;
    double *F = calloc((size_t)P->nt * N, sizeof(double));
    double *w = malloc(sizeof(double) * P->nt);
    or_ricker(P->nt, P->dt, P->f0, P->t0, w);
    size_t ps = src_node(P, s);
    for (int n = 0; n < P->nt; ++n) F[(size_t)n * N + ps] = w[n] / (P->h * P->h);
    solve_S(O, F, U);
    free(F); free(w);
}

/* P: sample receivers, d[n][r] = U[n][rec_r]. */
static void sample(const or_problem *P, int s, size_t N, const double *U, double *d)
{
    for (int n = 0; n < P->nt; ++n)
        for (int r = 0; r < P->nr; ++r)
            d[(size_t)n * P->nr + r] = U[(size_t)n * N + rec_node(P, s, r)];
}

/* P^T: spread receiver values into a dense unknown-space history. */
static void spread(const or_problem *P, int s, size_t N, const double *d, double *G)
{
    memset(G, 0, sizeof(double) * (size_t)P->nt * N);
    for (int n = 0; n < P->nt; ++n)
        for (int r = 0; r < P->nr; ++r)
            G[(size_t)n * N + rec_node(P, s, r)] += d[(size_t)n * P->nr + r];
}

/* Born data of one shot for an extended perturbation dmext (no noise weighting). */
static void shot_born(or_ops *O, const double *D, const double *dmext, int s, double *dd)
{
    const or_problem *P = O->P;
    size_t N = O->N;
    double *F = malloc(sizeof(double) * (size_t)P->nt * N);
    double *dU = malloc(sizeof(double) * (size_t)P->nt * N);
    for (int n = 0; n < P->nt; ++n)            /* (G dm)^n */
        for (size_t p = 0; p < N; ++p) {
            double mm = O->m[p];
            F[(size_t)n * N + p] = 2.0 * dmext[p] / (mm * mm * mm) * D[(size_t)n * N + p];
        }
    solve_S(O, F, dU);
    sample(P, s, N, dU, dd);
    free(F); free(dU);
}

/* Extended-grid image G^T S^{-T} P^T r of one shot (accumulated into img). */
static void shot_adjoint(or_ops *O, const double *D, const double *r, int s, double *img)
{
    const or_problem *P = O->P;
    size_t N = O->N;
    double *G = malloc(sizeof(double) * (size_t)P->nt * N);
    double *Lam = malloc(sizeof(double) * (size_t)P->nt * N);
    spread(P, s, N, r, G);
    solve_ST(O, G, Lam);
    for (size_t p = 0; p < N; ++p) {
        double mm = O->m[p];
        double acc = 0.0;
        for (int n = 0; n < P->nt; ++n)
            acc += Lam[(size_t)n * N + p] * D[(size_t)n * N + p];
        img[p] += 2.0 / (mm * mm * mm) * acc;
    }
    free(G); free(Lam);
}

/* ------------------------------------------------------------------------ */
/* Shot-parallel driver.  Every shot writes only its own slice; results that
 * sum over shots are summed afterwards in shot order, so the answer does not
 * depend on the thread count. */
typedef enum { JOB_FWD, JOB_BORN, JOB_ADJ, JOB_GRAD, JOB_HV } job_kind;

typedef struct {
    const or_problem *P;
    job_kind kind;
    const double *mext;
    const double *in;        /* BORN/HV: extended perturbations [k][N]; ADJ: r [ns][nt][nr]; GRAD: d_obs */
    int k;                   /* number of vectors (BORN/HV)                                  */
    double *out;             /* FWD/BORN: data; ADJ/GRAD/HV: per-shot images [ns][k][N]      */
    double *phi;             /* GRAD: per-shot misfits [ns]                                  */
    int next_shot;
    pthread_mutex_t lock;
    int failed;
} job;

static void run_shot(job *J, int s)
{
    const or_problem *P = J->P;
    or_ops O;
    if (ops_init(&O, P, J->mext) != 0) { J->failed = 1; return; }
    size_t N = O.N;
    size_t nd = (size_t)P->nt * P->nr;
    double *U = malloc(sizeof(double) * (size_t)P->nt * N);
    double *D = malloc(sizeof(double) * (size_t)P->nt * N);
    shot_forward(&O, s, U);
    if (J->kind == JOB_FWD) {
        sample(P, s, N, U, J->out + (size_t)s * nd);
    } else {
        time_operator(&O, U, D);
        if (J->kind == JOB_BORN) {
            for (int j = 0; j < J->k; ++j)
                shot_born(&O, D, J->in + (size_t)j * N, s, J->out + ((size_t)j * P->ns + s) * nd);
        } else if (J->kind == JOB_ADJ) {
            double *img = J->out + (size_t)s * N;
            memset(img, 0, sizeof(double) * N);
            shot_adjoint(&O, D, J->in + (size_t)s * nd, s, img);
        } else if (J->kind == JOB_GRAD) {
            double *d = malloc(sizeof(double) * nd);
            double *r = malloc(sizeof(double) * nd);
            sample(P, s, N, U, d);
            double is2 = 1.0 / (P->sigma * P->sigma), acc = 0.0;
            for (size_t i = 0; i < nd; ++i) {
                double res = d[i] - J->in[(size_t)s * nd + i];
                acc += res * res;
                r[i] = res * is2;
            }
            J->phi[s] = 0.5 * is2 * acc;
            double *img = J->out + (size_t)s * N;
            memset(img, 0, sizeof(double) * N);
            shot_adjoint(&O, D, r, s, img);
            free(d); free(r);
        } else { /* JOB_HV */
            double *dd = malloc(sizeof(double) * nd);
            double is2 = 1.0 / (P->sigma * P->sigma);
            for (int j = 0; j < J->k; ++j) {
                shot_born(&O, D, J->in + (size_t)j * N, s, dd);
                for (size_t i = 0; i < nd; ++i) dd[i] *= is2;          /* Gamma^{-1} */
                double *img = J->out + ((size_t)s * J->k + j) * N;
                memset(img, 0, sizeof(double) * N);
                shot_adjoint(&O, D, dd, s, img);
            }
            free(dd);
        }
    }
    free(U); free(D);
    ops_free(&O);
}

static void *worker(void *arg)
{
    job *J = arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int s = J->next_shot++;
        pthread_mutex_unlock(&J->lock);
        if (s >= J->P->ns) break;
        run_shot(J, s);
    }
    return NULL;
}

static int run_job(job *J, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > J->P->ns) nthreads = J->P->ns;
    J->next_shot = 0;
    J->failed = 0;
    pthread_mutex_init(&J->lock, NULL);
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J->lock);
    return J->failed ? -1 : 0;
}

static double *extend_new(const or_problem *P, const double *m)
{
    double *mext = malloc(sizeof(double) * (size_t)NZ_(P) * NX_(P));
    or_extend(P, m, mext);
    return mext;
}

/* Sum per-shot extended images in shot order and fold them to the interior. */
static void reduce_fold(const or_problem *P, const double *imgs, int k, int j, double *g)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *acc = calloc(N, sizeof(double));
    for (int s = 0; s < P->ns; ++s)
        for (size_t p = 0; p < N; ++p) acc[p] += imgs[((size_t)s * k + j) * N + p];
    or_fold(P, acc, g);
    free(acc);
}

/* ------------------------------------------------------------------------ */
/* Public entry points (all arrays are host, double, caller-owned). */

/* f(m): d[ns][nt][nr] (paper eq. (data) without noise). */
int or_fwd_model(const or_problem *P, const double *m, double *d, int nthreads)
{
    double *mext = extend_new(P, m);
    job J = {.P = P, .kind = JOB_FWD, .mext = mext, .out = d};
    int rc = run_job(&J, nthreads);
    free(mext);
    return rc;
}

/* Wavefield history of one shot on the padded grid: U[n] = u^{n+1}, n < nt. */
int or_wavefield(const or_problem *P, const double *m, int shot, double *U)
{
    double *mext = extend_new(P, m);
    or_ops O;
    if (ops_init(&O, P, mext) != 0) { free(mext); return -1; }
    shot_forward(&O, shot, U);
    ops_free(&O);
    free(mext);
    return 0;
}

/* Born (linearised) data F dm for k interior perturbations: dd[k][ns][nt][nr]. */
int or_born(const or_problem *P, const double *m, int k, const double *dm, double *dd, int nthreads)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *mext = extend_new(P, m);
    double *dmext = malloc(sizeof(double) * N * k);
    for (int j = 0; j < k; ++j) or_extend(P, dm + (size_t)j * P->nz * P->nx, dmext + (size_t)j * N);
    job J = {.P = P, .kind = JOB_BORN, .mext = mext, .in = dmext, .k = k, .out = dd};
    int rc = run_job(&J, nthreads);
    free(mext); free(dmext);
    return rc;
}

/* Migration F^T r (paper eq. (grad), F* applied to data r[ns][nt][nr]): g[nz][nx]. */
int or_adjoint(const or_problem *P, const double *m, const double *r, double *g, int nthreads)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *mext = extend_new(P, m);
    double *imgs = malloc(sizeof(double) * N * P->ns);
    job J = {.P = P, .kind = JOB_ADJ, .mext = mext, .in = r, .k = 1, .out = imgs};
    int rc = run_job(&J, nthreads);
    if (rc == 0) reduce_fold(P, imgs, 1, 0, g);
    free(mext); free(imgs);
    return rc;
}

/* Misfit Phi = (1/2 sigma^2) sum (f(m) - d_obs)^2 and its gradient F^T Gamma^{-1}(f(m) - d_obs). */
int or_misfit_grad(const or_problem *P, const double *m, const double *dobs, double *phi, double *g, int nthreads)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *mext = extend_new(P, m);
    double *imgs = malloc(sizeof(double) * N * P->ns);
    double *phis = malloc(sizeof(double) * P->ns);
    job J = {.P = P, .kind = JOB_GRAD, .mext = mext, .in = dobs, .k = 1, .out = imgs, .phi = phis};
    int rc = run_job(&J, nthreads);
    if (rc == 0) {
        double acc = 0.0;
        for (int s = 0; s < P->ns; ++s) acc += phis[s];
        *phi = acc;
        reduce_fold(P, imgs, 1, 0, g);
    }
    free(mext); free(imgs); free(phis);
    return rc;
}

/* Gauss-Newton Hessian apply, Hv[j] = F^T Gamma^{-1} F v[j], j < k (paper section 3). */
int or_hessian_apply(const or_problem *P, const double *m, int k, const double *v, double *Hv, int nthreads)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *mext = extend_new(P, m);
    double *vext = malloc(sizeof(double) * N * k);
    for (int j = 0; j < k; ++j) or_extend(P, v + (size_t)j * P->nz * P->nx, vext + (size_t)j * N);
    double *imgs = malloc(sizeof(double) * N * k * P->ns);
    job J = {.P = P, .kind = JOB_HV, .mext = mext, .in = vext, .k = k, .out = imgs};
    int rc = run_job(&J, nthreads);
    if (rc == 0)
        for (int j = 0; j < k; ++j) reduce_fold(P, imgs, k, j, Hv + (size_t)j * P->nz * P->nx);
    free(mext); free(vext); free(imgs);
    return rc;
}

/* The extended image before the fold E^T: ext[j] = sum over shots (in shot
 * order) of G^T S^-T P^T Gamma^-1 P S^-1 G E v[j] on the padded grid, so that
 * or_fold(ext[j]) is or_hessian_apply's Hv[j] (section 3, the sum over sources). */
int or_hessian_image(const or_problem *P, const double *m, int k, const double *v, double *ext, int nthreads)
{
    size_t N = (size_t)NZ_(P) * NX_(P);
    double *mext = extend_new(P, m);
    double *vext = malloc(sizeof(double) * N * k);
    for (int j = 0; j < k; ++j) or_extend(P, v + (size_t)j * P->nz * P->nx, vext + (size_t)j * N);
    double *imgs = malloc(sizeof(double) * N * k * P->ns);
    job J = {.P = P, .kind = JOB_HV, .mext = mext, .in = vext, .k = k, .out = imgs};
    int rc = run_job(&J, nthreads);
    if (rc == 0)
        for (int j = 0; j < k; ++j) {
            double *acc = ext + (size_t)j * N;
            memset(acc, 0, sizeof(double) * N);
            for (int s = 0; s < P->ns; ++s)
                for (size_t p = 0; p < N; ++p) acc[p] += imgs[((size_t)s * k + j) * N + p];
        }
    free(mext); free(vext); free(imgs);
    return rc;
}

/* Raw solves on the padded grid for the operator-level dot test
 * <S^{-1} F, G> = <F, S^{-T} G>: F, G, U, Lam are [nt][NZ*NX]. */
int or_solve_S(const or_problem *P, const double *m, const double *F, double *U)
{
    double *mext = extend_new(P, m);
    or_ops O;
    if (ops_init(&O, P, mext) != 0) { free(mext); return -1; }
    solve_S(&O, F, U);
    ops_free(&O);
    free(mext);
    return 0;
}

int or_solve_ST(const or_problem *P, const double *m, const double *G, double *Lam)
{
    double *mext = extend_new(P, m);
    or_ops O;
    if (ops_init(&O, P, mext) != 0) { free(mext); return -1; }
    solve_ST(&O, G, Lam);
    ops_free(&O);
    free(mext);
    return 0;
}
