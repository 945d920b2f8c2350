/*
 * fdtd_oracle.c -- FP64 CPU oracle of the 3D Yee FDTD near-field path.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code, header, table or constant generator with the CUDA library; the two
 * meet only through the seeded inputs of workloads.py.
 *
 * What it computes, step n -> n+1 (E^0 = 0, H^{-1/2} = 0):
 *   1. H^{n+1/2} = H^{n-1/2} - (dt/mu0) curl E^n              (Sec. III.A, the
 *      Maxwell curl equations and the Yee leapfrog), CPML psi_H first;
 *   2. the current J_z^{n+1/2} of the net charge excess moving along the axis
 *      (Sec. III.B, shower model; Sec. I, 20% charge excess);
 *   3. E^{n+1} = E^n + (dt/eps) curl H^{n+1/2} - (dt/eps) J,     CPML psi_E;
 *   4. first-order Mur on the tangential E of the six faces, or PEC;
 *   5. detectors record E at fixed points (Sec. III.B, "Simulation Setup").
 * The paper is silent on the boundary, the deposit, the update order in 3D
 * and dt.  Readings taken here: the leapfrog runs H^{n+1/2} then E^{n+1} from
 * E^0 = H^{-1/2} = 0 (the paper's E-then-H order with shifted labels);
 * dt = 0.5 dx sqrt(eps_r) / (c sqrt 3); the boundary is first-order Mur
 * (apply_mur) or a Roden-Gedney CPML with PEC behind it (cpml_coef); the charge
 * moves as a cloud-in-cell line whose current carries exactly the charge that
 * crossed each face, and changes of the profile are charge created or lost at
 * rest (build_source).
 *
 * Plain loops, no blocking, compiled with -ffp-contract=off.  The only
 * parallelism is an OpenMP loop over independent cells (bitwise
 * deterministic: no reductions).
 *
 * Layout: every component lives on the node grid (nx+1)(ny+1)(nz+1), x
 * fastest; index (i,j,k) holds
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k);
 * entries outside a component's range stay zero.
 *
 * Parity pins: tests/test_oracle_*.py (dispersion, cavity modes, energy,
 * Gauss law, dipole closed form, Cherenkov angle, boundary reflection).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PEC 0
#define ORC_MUR1 1
#define ORC_CPML 2

static const double ORC_C0 = 299792458.0;         /* m/s, exact */
static const double ORC_MU0 = 1.25663706212e-6;   /* H/m, CODATA 2018 */

typedef struct orc {
    int nx, ny, nz, bc, P;
    double dx, dt, eps_r, eps, kE, kH;
    size_t nn;
    double *f[6];      /* Ex Ey Ez Hx Hy Hz */
    double *eold[3];   /* E^n kept for the Mur faces */
    /* CPML coefficients per axis: E-type (integer position) and H-type
       (half-integer position) a, b indexed by the position index. */
    double *aE[3], *bE[3], *aH[3], *bH[3];
    /* psi arrays, stored over the two slabs of their axis only:
       x: [nz+1][ny+1][2P]   y: [nz+1][2P][nx+1]   z: [2P][ny+1][nx+1]   */
    double *psi_eyx, *psi_ezx, *psi_hyx, *psi_hzx;
    double *psi_exy, *psi_ezy, *psi_hxy, *psi_hzy;
    double *psi_exz, *psi_eyz, *psi_hxz, *psi_hyz;
    /* source */
    int has_src, L, nbins;
    double *q, z0, bin_dz, v, *w;
    int ic, jc;
    /* last step's source entries: node-grid index of Ez and J_z value */
    int nsrc;
    size_t *src_idx;
    double *src_j;
    /* probes */
    int np, max_steps;
    int *pi, *pj, *pk;
    double *trace; /* [np][max_steps][2] */
    long step;
} orc;

static size_t ID(const orc *o, int i, int j, int k) {
    return ((size_t)k * (size_t)(o->ny + 1) + (size_t)j) * (size_t)(o->nx + 1) + (size_t)i;
}

/* Index of a position inside the two PML slabs of an axis with N cells, or -1.
   E-type positions are the integers 1..P and N-P..N-1; H-type positions are
   the half-integers i+1/2 for i in 0..P-1 and N-P..N-1. */
static int slab_e(int i, int N, int P) {
    if (P <= 0) return -1;
    if (i >= 1 && i <= P) return i - 1;
    if (i >= N - P && i <= N - 1) return i - (N - 2 * P);
    return -1;
}
static int slab_h(int i, int N, int P) {
    if (P <= 0) return -1;
    if (i >= 0 && i <= P - 1) return i;
    if (i >= N - P && i <= N - 1) return i - (N - 2 * P);
    return -1;
}

double orc_c0(void) { return ORC_C0; }
double orc_mu0(void) { return ORC_MU0; }
double orc_eps0(void) { return 1.0 / (ORC_MU0 * ORC_C0 * ORC_C0); }

/* Roden-Gedney CPML grading (reading of the paper's silence on the boundary):
   sigma(d) = sigma_max (d/P)^3, sigma_max = -(m+1) ln(R0) / (2 eta P dx),
   eta = eta0/sqrt(eps_r), R0 = 1e-6; kappa = 1; alpha falls linearly from
   2 pi 50 MHz eps at the interface (d = 0) to 0 at the outer PEC wall (d = P);
   b = exp(-(sigma + alpha) dt / eps), a = sigma (b - 1) / (sigma + alpha). */
static void cpml_coef(const orc *o, double d, double *a, double *b) {
    const double m = 3.0, R0 = 1e-6;
    double eta = ORC_MU0 * ORC_C0 / sqrt(o->eps_r);
    double smax = -(m + 1.0) * log(R0) / (2.0 * eta * o->P * o->dx);
    double amax = 2.0 * M_PI * 50e6 * o->eps;
    double s = smax * pow(d / o->P, m);
    double al = amax * (1.0 - d / o->P);
    *b = exp(-(s + al) * o->dt / o->eps);
    *a = (s + al) > 0.0 ? s * (*b - 1.0) / (s + al) : 0.0;
}

static void orc_free(orc *o) {
    if (!o) return;
    for (int c = 0; c < 6; ++c) free(o->f[c]);
    for (int c = 0; c < 3; ++c) {
        free(o->eold[c]);
        free(o->aE[c]); free(o->bE[c]); free(o->aH[c]); free(o->bH[c]);
    }
    free(o->psi_eyx); free(o->psi_ezx); free(o->psi_hyx); free(o->psi_hzx);
    free(o->psi_exy); free(o->psi_ezy); free(o->psi_hxy); free(o->psi_hzy);
    free(o->psi_exz); free(o->psi_eyz); free(o->psi_hxz); free(o->psi_hyz);
    free(o->q); free(o->w); free(o->src_idx); free(o->src_j);
    free(o->pi); free(o->pj); free(o->pk); free(o->trace);
    free(o);
}

void orc_destroy(orc *o) { orc_free(o); }

/* Returns NULL on bad arguments or when memory runs out. */
orc *orc_create(int nx, int ny, int nz, double dx, double dt, double eps_r,
                int bc, int npml) {
    if (nx < 4 || ny < 4 || nz < 4 || !(dx > 0) || !(dt > 0) || !(eps_r >= 1))
        return NULL;
    if (bc != ORC_PEC && bc != ORC_MUR1 && bc != ORC_CPML) return NULL;
    if (bc == ORC_CPML) {
        if (npml < 1 || nx < 2 * npml + 4 || ny < 2 * npml + 4 || nz < 2 * npml + 4)
            return NULL;
    } else {
        npml = 0;
    }
    orc *o = (orc *)calloc(1, sizeof(orc));
    if (!o) return NULL;
    o->nx = nx; o->ny = ny; o->nz = nz; o->bc = bc; o->P = npml;
    o->dx = dx; o->dt = dt; o->eps_r = eps_r;
    o->eps = eps_r / (ORC_MU0 * ORC_C0 * ORC_C0);
    o->kE = dt / (o->eps * dx);
    o->kH = dt / (ORC_MU0 * dx);
    o->nn = (size_t)(nx + 1) * (size_t)(ny + 1) * (size_t)(nz + 1);
    for (int c = 0; c < 6; ++c) {
        o->f[c] = (double *)calloc(o->nn, sizeof(double));
        if (!o->f[c]) { orc_free(o); return NULL; }
    }
    if (bc == ORC_MUR1) {
        for (int c = 0; c < 3; ++c) {
            o->eold[c] = (double *)calloc(o->nn, sizeof(double));
            if (!o->eold[c]) { orc_free(o); return NULL; }
        }
    }
    if (bc == ORC_CPML) {
        int N[3] = {nx, ny, nz};
        for (int ax = 0; ax < 3; ++ax) {
            int n = N[ax];
            o->aE[ax] = (double *)calloc(n + 1, sizeof(double));
            o->bE[ax] = (double *)calloc(n + 1, sizeof(double));
            o->aH[ax] = (double *)calloc(n + 1, sizeof(double));
            o->bH[ax] = (double *)calloc(n + 1, sizeof(double));
            if (!o->aE[ax] || !o->bE[ax] || !o->aH[ax] || !o->bH[ax]) { orc_free(o); return NULL; }
            for (int i = 0; i <= n; ++i) {
                double d;
                if (slab_e(i, n, npml) >= 0) {
                    d = (i <= npml) ? (double)(npml - i) : (double)(i - (n - npml));
                    cpml_coef(o, d, &o->aE[ax][i], &o->bE[ax][i]);
                }
                if (i < n && slab_h(i, n, npml) >= 0) {
                    d = (i < npml) ? (npml - i - 0.5) : (i + 0.5 - (n - npml));
                    cpml_coef(o, d, &o->aH[ax][i], &o->bH[ax][i]);
                }
            }
        }
        size_t px = (size_t)(nz + 1) * (ny + 1) * 2 * npml;
        size_t py = (size_t)(nz + 1) * 2 * npml * (nx + 1);
        size_t pz = (size_t)2 * npml * (ny + 1) * (nx + 1);
        double **xs[4] = {&o->psi_eyx, &o->psi_ezx, &o->psi_hyx, &o->psi_hzx};
        double **ys[4] = {&o->psi_exy, &o->psi_ezy, &o->psi_hxy, &o->psi_hzy};
        double **zs[4] = {&o->psi_exz, &o->psi_eyz, &o->psi_hxz, &o->psi_hyz};
        for (int t = 0; t < 4; ++t) {
            *xs[t] = (double *)calloc(px, sizeof(double));
            *ys[t] = (double *)calloc(py, sizeof(double));
            *zs[t] = (double *)calloc(pz, sizeof(double));
            if (!*xs[t] || !*ys[t] || !*zs[t]) { orc_free(o); return NULL; }
        }
    }
    o->ic = nx / 2;
    o->jc = ny / 2;
    return o;
}

static size_t PX(const orc *o, int l, int j, int k) {
    return ((size_t)k * (o->ny + 1) + j) * (size_t)(2 * o->P) + l;
}
static size_t PY(const orc *o, int i, int l, int k) {
    return ((size_t)k * (2 * o->P) + l) * (size_t)(o->nx + 1) + i;
}
static size_t PZ(const orc *o, int i, int j, int l) {
    return ((size_t)l * (o->ny + 1) + j) * (size_t)(o->nx + 1) + i;
}

/* Source: Q(z) is a table of samples q[b] at z0 + b*bin_dz, interpolated
   linearly and zero outside the table; the charge moves along the node line
   (nx/2, ny/2) with speed v, entering at z0 at step 0; w is the
   (2L+1)x(2L+1) lateral weight table, w[(dj+L)(2L+1) + (di+L)]. */
int orc_set_shower(orc *o, const double *q, int nbins, double z0, double bin_dz,
                   double v, const double *w, int L) {
    if (!o || !q || !w || nbins < 2 || !(bin_dz > 0) || L < 0) return -1;
    int lo = o->bc == ORC_CPML ? o->P + 1 : 1;
    if (o->ic - L < lo || o->ic + L > o->nx - lo) return -1;
    if (o->jc - L < lo || o->jc + L > o->ny - lo) return -1;
    free(o->q); free(o->w); free(o->src_idx); free(o->src_j);
    int nw = (2 * L + 1) * (2 * L + 1);
    o->q = (double *)malloc(sizeof(double) * nbins);
    o->w = (double *)malloc(sizeof(double) * nw);
    /* a step touches at most ceil(|v| dt/dx) + 2 edges per footprint column */
    int nk = (int)ceil(fabs(v) * o->dt / o->dx) + 2;
    o->src_idx = (size_t *)malloc(sizeof(size_t) * (size_t)nw * nk);
    o->src_j = (double *)malloc(sizeof(double) * (size_t)nw * nk);
    if (!o->q || !o->w || !o->src_idx || !o->src_j) return -2;
    memcpy(o->q, q, sizeof(double) * nbins);
    memcpy(o->w, w, sizeof(double) * nw);
    o->nbins = nbins; o->z0 = z0; o->bin_dz = bin_dz; o->v = v; o->L = L;
    o->has_src = 1;
    o->nsrc = 0;
    return 0;
}

double orc_profile_at(const orc *o, double z) {
    double u = (z - o->z0) / o->bin_dz;
    if (!(u >= 0.0) || u > (double)(o->nbins - 1)) return 0.0;
    int b = (int)floor(u);
    if (b >= o->nbins - 1) return o->q[o->nbins - 1];
    double t = u - b;
    return o->q[b] * (1.0 - t) + o->q[b + 1] * t;
}

/* Fraction of a unit charge at height z (metres) that the linear (CIC) hat
   puts on nodes k' <= k of the untruncated line: 0, 1-f or 1. */
static double cum_cic(double z, double dx, int k) {
    double u = z / dx;
    double k0 = floor(u);
    double f = u - k0;
    if ((double)k < k0) return 0.0;
    if ((double)k == k0) return 1.0 - f;
    return 1.0;
}

/* Probes: positions in metres from node (0,0,0), snapped to the nearest node,
   which must lie inside the non-PML interior with one node of margin. */
int orc_set_probes(orc *o, const double *xyz, int n, int max_steps) {
    if (!o || n < 0 || max_steps < 0 || (n > 0 && !xyz)) return -1;
    free(o->pi); free(o->pj); free(o->pk); free(o->trace);
    o->pi = o->pj = o->pk = NULL; o->trace = NULL;
    o->np = 0; o->max_steps = max_steps;
    if (n == 0) return 0;
    o->pi = (int *)malloc(sizeof(int) * n);
    o->pj = (int *)malloc(sizeof(int) * n);
    o->pk = (int *)malloc(sizeof(int) * n);
    o->trace = (double *)calloc((size_t)n * (size_t)(max_steps > 0 ? max_steps : 1) * 2, sizeof(double));
    if (!o->pi || !o->pj || !o->pk || !o->trace) return -2;
    int lo = o->bc == ORC_CPML ? o->P + 1 : 1;
    for (int p = 0; p < n; ++p) {
        int i = (int)floor(xyz[3 * p + 0] / o->dx + 0.5);
        int j = (int)floor(xyz[3 * p + 1] / o->dx + 0.5);
        int k = (int)floor(xyz[3 * p + 2] / o->dx + 0.5);
        if (i < lo || i > o->nx - lo || j < lo || j > o->ny - lo || k < lo || k > o->nz - lo)
            return -1;
        o->pi[p] = i; o->pj[p] = j; o->pk[p] = k;
    }
    o->np = n;
    return 0;
}

static void update_h(orc *o) {
    const int nx = o->nx, ny = o->ny, nz = o->nz, P = o->P;
    const int pml = o->bc == ORC_CPML;
    double *Ex = o->f[0], *Ey = o->f[1], *Ez = o->f[2];
    double *Hx = o->f[3], *Hy = o->f[4], *Hz = o->f[5];
    const double kH = o->kH;

    /* Hx(i, j+1/2, k+1/2) -= kH [ (Ez(j+1) - Ez(j)) - (Ey(k+1) - Ey(k)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                double dy = Ez[ID(o, i, j + 1, k)] - Ez[ID(o, i, j, k)];
                double dz = Ey[ID(o, i, j, k + 1)] - Ey[ID(o, i, j, k)];
                if (pml) {
                    int l = slab_h(j, ny, P);
                    if (l >= 0) {
                        double *p = &o->psi_hxy[PY(o, i, l, k)];
                        *p = o->bH[1][j] * (*p) + o->aH[1][j] * dy;
                        dy = dy + *p;
                    }
                    l = slab_h(k, nz, P);
                    if (l >= 0) {
                        double *p = &o->psi_hxz[PZ(o, i, j, l)];
                        *p = o->bH[2][k] * (*p) + o->aH[2][k] * dz;
                        dz = dz + *p;
                    }
                }
                Hx[ID(o, i, j, k)] -= kH * (dy - dz);
            }

    /* Hy(i+1/2, j, k+1/2) -= kH [ (Ex(k+1) - Ex(k)) - (Ez(i+1) - Ez(i)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double dz = Ex[ID(o, i, j, k + 1)] - Ex[ID(o, i, j, k)];
                double dx = Ez[ID(o, i + 1, j, k)] - Ez[ID(o, i, j, k)];
                if (pml) {
                    int l = slab_h(k, nz, P);
                    if (l >= 0) {
                        double *p = &o->psi_hyz[PZ(o, i, j, l)];
                        *p = o->bH[2][k] * (*p) + o->aH[2][k] * dz;
                        dz = dz + *p;
                    }
                    l = slab_h(i, nx, P);
                    if (l >= 0) {
                        double *p = &o->psi_hyx[PX(o, l, j, k)];
                        *p = o->bH[0][i] * (*p) + o->aH[0][i] * dx;
                        dx = dx + *p;
                    }
                }
                Hy[ID(o, i, j, k)] -= kH * (dz - dx);
            }

    /* Hz(i+1/2, j+1/2, k) -= kH [ (Ey(i+1) - Ey(i)) - (Ex(j+1) - Ex(j)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double dx = Ey[ID(o, i + 1, j, k)] - Ey[ID(o, i, j, k)];
                double dy = Ex[ID(o, i, j + 1, k)] - Ex[ID(o, i, j, k)];
                if (pml) {
                    int l = slab_h(i, nx, P);
                    if (l >= 0) {
                        double *p = &o->psi_hzx[PX(o, l, j, k)];
                        *p = o->bH[0][i] * (*p) + o->aH[0][i] * dx;
                        dx = dx + *p;
                    }
                    l = slab_h(j, ny, P);
                    if (l >= 0) {
                        double *p = &o->psi_hzy[PY(o, i, l, k)];
                        *p = o->bH[1][j] * (*p) + o->aH[1][j] * dy;
                        dy = dy + *p;
                    }
                }
                Hz[ID(o, i, j, k)] -= kH * (dx - dy);
            }
}

/* J_z^{n+1/2} on the Ez edges (i, j, k+1/2) of the footprint: the charge
   qbar = Q(z_s^{n+1/2}) moves from z_s^n to z_s^{n+1}; the current through
   edge k+1/2 is the charge that crossed it,
       J = -(dx/dt) qbar w_ij / dx^3 [C_k(z^{n+1}) - C_k(z^n)],
   C_k = cumulative CIC weight on nodes <= k of the untruncated line.  The
   current is kept on edges outside the PML only (all edges for Mur/PEC). */
static void build_source(orc *o) {
    o->nsrc = 0;
    if (!o->has_src) return;
    const double dx = o->dx, dt = o->dt;
    double z0 = o->z0 + o->v * (double)o->step * dt;
    double z1 = o->z0 + o->v * (double)(o->step + 1) * dt;
    double qbar = orc_profile_at(o, o->z0 + o->v * ((double)o->step + 0.5) * dt);
    if (qbar == 0.0) return;
    int klo = (int)floor(fmin(z0, z1) / dx) - 1;
    int khi = (int)floor(fmax(z0, z1) / dx) + 1;
    int kmin = o->bc == ORC_CPML ? o->P : 0;
    int kmax = o->bc == ORC_CPML ? o->nz - o->P - 1 : o->nz - 1;
    int L = o->L;
    for (int k = klo; k <= khi; ++k) {
        if (k < kmin || k > kmax) continue;
        double dC = cum_cic(z1, dx, k) - cum_cic(z0, dx, k);
        if (dC == 0.0) continue;
        for (int dj = -L; dj <= L; ++dj)
            for (int di = -L; di <= L; ++di) {
                double wij = o->w[(dj + L) * (2 * L + 1) + (di + L)];
                if (wij == 0.0) continue;
                double J = -(dx / dt) * qbar * wij / (dx * dx * dx) * dC;
                o->src_idx[o->nsrc] = ID(o, o->ic + di, o->jc + dj, k);
                o->src_j[o->nsrc] = J;
                o->nsrc++;
            }
    }
}

static void update_e(orc *o) {
    const int nx = o->nx, ny = o->ny, nz = o->nz, P = o->P;
    const int pml = o->bc == ORC_CPML;
    double *Ex = o->f[0], *Ey = o->f[1], *Ez = o->f[2];
    double *Hx = o->f[3], *Hy = o->f[4], *Hz = o->f[5];
    const double kE = o->kE;

    /* Ex(i+1/2, j, k) += kE [ (Hz(j) - Hz(j-1)) - (Hy(k) - Hy(k-1)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double dy = Hz[ID(o, i, j, k)] - Hz[ID(o, i, j - 1, k)];
                double dz = Hy[ID(o, i, j, k)] - Hy[ID(o, i, j, k - 1)];
                if (pml) {
                    int l = slab_e(j, ny, P);
                    if (l >= 0) {
                        double *p = &o->psi_exy[PY(o, i, l, k)];
                        *p = o->bE[1][j] * (*p) + o->aE[1][j] * dy;
                        dy = dy + *p;
                    }
                    l = slab_e(k, nz, P);
                    if (l >= 0) {
                        double *p = &o->psi_exz[PZ(o, i, j, l)];
                        *p = o->bE[2][k] * (*p) + o->aE[2][k] * dz;
                        dz = dz + *p;
                    }
                }
                Ex[ID(o, i, j, k)] += kE * (dy - dz);
            }

    /* Ey(i, j+1/2, k) += kE [ (Hx(k) - Hx(k-1)) - (Hz(i) - Hz(i-1)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                double dz = Hx[ID(o, i, j, k)] - Hx[ID(o, i, j, k - 1)];
                double dx = Hz[ID(o, i, j, k)] - Hz[ID(o, i - 1, j, k)];
                if (pml) {
                    int l = slab_e(k, nz, P);
                    if (l >= 0) {
                        double *p = &o->psi_eyz[PZ(o, i, j, l)];
                        *p = o->bE[2][k] * (*p) + o->aE[2][k] * dz;
                        dz = dz + *p;
                    }
                    l = slab_e(i, nx, P);
                    if (l >= 0) {
                        double *p = &o->psi_eyx[PX(o, l, j, k)];
                        *p = o->bE[0][i] * (*p) + o->aE[0][i] * dx;
                        dx = dx + *p;
                    }
                }
                Ey[ID(o, i, j, k)] += kE * (dz - dx);
            }

    /* Ez(i, j, k+1/2) += kE [ (Hy(i) - Hy(i-1)) - (Hx(j) - Hx(j-1)) ] */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                double dx = Hy[ID(o, i, j, k)] - Hy[ID(o, i - 1, j, k)];
                double dy = Hx[ID(o, i, j, k)] - Hx[ID(o, i, j - 1, k)];
                if (pml) {
                    int l = slab_e(i, nx, P);
                    if (l >= 0) {
                        double *p = &o->psi_ezx[PX(o, l, j, k)];
                        *p = o->bE[0][i] * (*p) + o->aE[0][i] * dx;
                        dx = dx + *p;
                    }
                    l = slab_e(j, ny, P);
                    if (l >= 0) {
                        double *p = &o->psi_ezy[PY(o, i, l, k)];
                        *p = o->bE[1][j] * (*p) + o->aE[1][j] * dy;
                        dy = dy + *p;
                    }
                }
                Ez[ID(o, i, j, k)] += kE * (dx - dy);
            }

    /* the moving charge's current: E -= (dt/eps) J */
    for (int s = 0; s < o->nsrc; ++s)
        Ez[o->src_idx[s]] -= (o->dt / o->eps) * o->src_j[s];
}

/* First-order Mur on the tangential E of each face:
     E_0^{n+1} = E_1^n + m (E_1^{n+1} - E_0^n),  m = (S-1)/(S+1),  S = c' dt/dx,
   where E_1 is the next node inward along the face normal.  Only face nodes
   whose inward neighbour is an interior-updated value are treated; the
   components on the twelve edges stay zero (PEC), so the faces do not depend
   on one another. */
static void apply_mur(orc *o) {
    const int nx = o->nx, ny = o->ny, nz = o->nz;
    double S = ORC_C0 / sqrt(o->eps_r) * o->dt / o->dx;
    double m = (S - 1.0) / (S + 1.0);
    double *E[3] = {o->f[0], o->f[1], o->f[2]};
    double **Eo = o->eold;
    /* x faces: Ey (j 0..ny-1, k 1..nz-1), Ez (j 1..ny-1, k 0..nz-1) */
    for (int s = 0; s < 2; ++s) {
        int i0 = s == 0 ? 0 : nx, i1 = s == 0 ? 1 : nx - 1;
        for (int k = 1; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                E[1][ID(o, i0, j, k)] = Eo[1][ID(o, i1, j, k)] +
                    m * (E[1][ID(o, i1, j, k)] - Eo[1][ID(o, i0, j, k)]);
        for (int k = 0; k < nz; ++k)
            for (int j = 1; j < ny; ++j)
                E[2][ID(o, i0, j, k)] = Eo[2][ID(o, i1, j, k)] +
                    m * (E[2][ID(o, i1, j, k)] - Eo[2][ID(o, i0, j, k)]);
    }
    /* y faces: Ex (i 0..nx-1, k 1..nz-1), Ez (i 1..nx-1, k 0..nz-1) */
    for (int s = 0; s < 2; ++s) {
        int j0 = s == 0 ? 0 : ny, j1 = s == 0 ? 1 : ny - 1;
        for (int k = 1; k < nz; ++k)
            for (int i = 0; i < nx; ++i)
                E[0][ID(o, i, j0, k)] = Eo[0][ID(o, i, j1, k)] +
                    m * (E[0][ID(o, i, j1, k)] - Eo[0][ID(o, i, j0, k)]);
        for (int k = 0; k < nz; ++k)
            for (int i = 1; i < nx; ++i)
                E[2][ID(o, i, j0, k)] = Eo[2][ID(o, i, j1, k)] +
                    m * (E[2][ID(o, i, j1, k)] - Eo[2][ID(o, i, j0, k)]);
    }
    /* z faces: Ex (i 0..nx-1, j 1..ny-1), Ey (i 1..nx-1, j 0..ny-1) */
    for (int s = 0; s < 2; ++s) {
        int k0 = s == 0 ? 0 : nz, k1 = s == 0 ? 1 : nz - 1;
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                E[0][ID(o, i, j, k0)] = Eo[0][ID(o, i, j, k1)] +
                    m * (E[0][ID(o, i, j, k1)] - Eo[0][ID(o, i, j, k0)]);
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i)
                E[1][ID(o, i, j, k0)] = Eo[1][ID(o, i, j, k1)] +
                    m * (E[1][ID(o, i, j, k1)] - Eo[1][ID(o, i, j, k0)]);
    }
}

/* Detector readout at node (i,j,k): E averaged onto the node (two-point means
   of the staggered samples), E_r = (X Ex + Y Ey)/r about the shower axis
   (0 on the axis), stored as (Ez, E_r) in slot n for the fields E^{n+1}. */
static void record_probes(orc *o) {
    if (o->np == 0 || o->step >= o->max_steps) return;
    const double dx = o->dx;
    for (int p = 0; p < o->np; ++p) {
        int i = o->pi[p], j = o->pj[p], k = o->pk[p];
        double ex = 0.5 * (o->f[0][ID(o, i - 1, j, k)] + o->f[0][ID(o, i, j, k)]);
        double ey = 0.5 * (o->f[1][ID(o, i, j - 1, k)] + o->f[1][ID(o, i, j, k)]);
        double ez = 0.5 * (o->f[2][ID(o, i, j, k - 1)] + o->f[2][ID(o, i, j, k)]);
        double X = (i - o->ic) * dx, Y = (j - o->jc) * dx;
        double r = sqrt(X * X + Y * Y);
        double er = r > 0.0 ? (X * ex + Y * ey) / r : 0.0;
        double *t = o->trace + ((size_t)p * o->max_steps + (size_t)o->step) * 2;
        t[0] = ez;
        t[1] = er;
    }
}

int orc_step(orc *o, int n) {
    if (!o || n < 0) return -1;
    for (int s = 0; s < n; ++s) {
        update_h(o);
        if (o->bc == ORC_MUR1)
            for (int c = 0; c < 3; ++c) memcpy(o->eold[c], o->f[c], sizeof(double) * o->nn);
        build_source(o);
        update_e(o);
        if (o->bc == ORC_MUR1) apply_mur(o);
        record_probes(o); /* slot n holds E^{n+1} */
        o->step++;
    }
    return 0;
}

long orc_steps_done(const orc *o) { return o->step; }

void orc_get_field(const orc *o, int c, double *out) { memcpy(out, o->f[c], sizeof(double) * o->nn); }
void orc_set_field(orc *o, int c, const double *in) { memcpy(o->f[c], in, sizeof(double) * o->nn); }
void orc_get_probes(const orc *o, double *out) {
    if (o->np > 0) memcpy(out, o->trace, sizeof(double) * (size_t)o->np * o->max_steps * 2);
}
void orc_get_probe_nodes(const orc *o, int *ijk) {
    for (int p = 0; p < o->np; ++p) {
        ijk[3 * p] = o->pi[p]; ijk[3 * p + 1] = o->pj[p]; ijk[3 * p + 2] = o->pk[p];
    }
}
/* The J_z entries injected by the last step: count, node-grid index, value. */
int orc_source_count(const orc *o) { return o->nsrc; }
void orc_get_source(const orc *o, int64_t *idx, double *val) {
    for (int s = 0; s < o->nsrc; ++s) { idx[s] = (int64_t)o->src_idx[s]; val[s] = o->src_j[s]; }
}
double orc_kE(const orc *o) { return o->kE; }
double orc_kH(const orc *o) { return o->kH; }
double orc_eps(const orc *o) { return o->eps; }
void orc_cpml_coefs(const orc *o, int axis, double *aE, double *bE, double *aH, double *bH) {
    int n = axis == 0 ? o->nx : axis == 1 ? o->ny : o->nz;
    for (int i = 0; i <= n; ++i) {
        aE[i] = o->aE[axis] ? o->aE[axis][i] : 0.0;
        bE[i] = o->bE[axis] ? o->bE[axis][i] : 0.0;
        aH[i] = o->aH[axis] ? o->aH[axis][i] : 0.0;
        bH[i] = o->bH[axis] ? o->bH[axis][i] : 0.0;
    }
}

/* ------------------------------------------------------------------------
 * Shower model tables (Sec. III.B).  Q(z) = -e f N_e(z) in coulombs.
 * ------------------------------------------------------------------------ */
static const double ORC_QE = 1.602176634e-19;

/* Eq. (showerModel): N_e(z) = N_max exp(-(z - z_peak)^2 / (2 l^2)); the table
   stores the charge q_max exp(...) directly. */
void orc_profile_gaussian(double z0, double bin_dz, int nbins, double z_peak,
                          double l, double q_max, double *out) {
    for (int b = 0; b < nbins; ++b) {
        double z = z0 + b * bin_dz;
        out[b] = q_max * exp(-(z - z_peak) * (z - z_peak) / (2.0 * l * l));
    }
}

/* Eq. (nkg_formula), the Greisen longitudinal profile, with the standard age
   s = 3t/(t + 2 beta0) (the printed age is garbled; this reading puts s = 1 at
   the maximum t = beta0): N_e(t) = 0.31/sqrt(beta0) exp[t (1 - 1.5 ln s)],
   t = (z - z0)/X0 in radiation lengths, beta0 = ln(E0/Ec). */
double orc_greisen(double t, double E0, double Ec) {
    if (!(t > 0.0)) return 0.0;
    double beta0 = log(E0 / Ec);
    double s = 3.0 * t / (t + 2.0 * beta0);
    return 0.31 / sqrt(beta0) * exp(t * (1.0 - 1.5 * log(s)));
}

void orc_profile_greisen(double z0, double bin_dz, int nbins, double E0, double Ec,
                         double X0, double frac, double *out) {
    (void)z0; /* the table starts at the first interaction, t = 0 */
    for (int b = 0; b < nbins; ++b) {
        double t = (b * bin_dz) / X0;
        out[b] = -ORC_QE * frac * orc_greisen(t, E0, Ec);
    }
}

/* Gaisser-Hillas subshowers (not in the paper; used to build an elongated,
   multi-peaked profile):
   N(z) = N_max ((z-z1)/(zm-z1))^((zm-z1)/lam) exp((zm - z)/lam) for z > z1. */
void orc_profile_gh(double z0, double bin_dz, int nbins, int nsub, const double *z1,
                    const double *zmax, const double *lam, const double *nmax,
                    double frac, double *out) {
    for (int b = 0; b < nbins; ++b) {
        double z = z0 + b * bin_dz, n = 0.0;
        for (int s = 0; s < nsub; ++s) {
            if (z <= z1[s]) continue;
            double w = zmax[s] - z1[s];
            n += nmax[s] * pow((z - z1[s]) / w, w / lam[s]) * exp((zmax[s] - z) / lam[s]);
        }
        out[b] = -ORC_QE * frac * n;
    }
}

/* Lateral weights on the (2L+1)^2 nodes around the axis, normalised to sum 1.
   Gaussian: w ~ exp(-(di^2 + dj^2) / (2 sigma^2)), sigma in cells, point values. */
void orc_lateral_gaussian(int L, double sigma_cells, double *w) {
    int n = 2 * L + 1;
    double sum = 0.0;
    for (int dj = -L; dj <= L; ++dj)
        for (int di = -L; di <= L; ++di) {
            double v = exp(-(double)(di * di + dj * dj) / (2.0 * sigma_cells * sigma_cells));
            w[(dj + L) * n + (di + L)] = v;
            sum += v;
        }
    for (int t = 0; t < n * n; ++t) w[t] /= sum;
}

/* NKG lateral density rho(r) ~ (r/rM)^(s-2) (1 + r/rM)^(s-4.5), averaged over
   nsub x nsub points of each node's cell, zero beyond r_cut, normalised. */
void orc_lateral_nkg(int L, double dx, double rM, double s, int nsub, double r_cut,
                     double *w) {
    int n = 2 * L + 1;
    double sum = 0.0;
    for (int dj = -L; dj <= L; ++dj)
        for (int di = -L; di <= L; ++di) {
            double acc = 0.0;
            for (int b = 0; b < nsub; ++b)
                for (int a = 0; a < nsub; ++a) {
                    double x = (di - 0.5 + (a + 0.5) / nsub) * dx;
                    double y = (dj - 0.5 + (b + 0.5) / nsub) * dx;
                    double r = sqrt(x * x + y * y);
                    if (r > r_cut || r <= 0.0) continue;
                    acc += pow(r / rM, s - 2.0) * pow(1.0 + r / rM, s - 4.5);
                }
            w[(dj + L) * n + (di + L)] = acc;
            sum += acc;
        }
    for (int t = 0; t < n * n; ++t) w[t] /= sum;
}

/* Threads of the oracle's parallel loops from now on (n >= 1), or unchanged
   for n <= 0; returns the count in force.  1 without OpenMP. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
