/*
 * mhs_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * linear magnetohydrostatic (MHS) multigrid path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library includes, links or
 * calls this file; the tests, the smoke check and the CPU-baseline leg of the
 * benchmark are its only users.  It shares no code with the CUDA path.
 *
 * What it computes (MacTaggart et al., "Non-symmetric magnetohydrostatic
 * equilibria: a multigrid approach"):
 *   - Sect. 2.2, eq. (lower_bound): P_xx + P_yy = -B_z on z = 0, P = 0 on the
 *     edges of the plane;
 *   - Sect. 2.1, eq. (scalar_pot): [1 - xi(z)](P_xx + P_yy) + P_zz + alpha^2 P = 0
 *     in the interior, P from the lower-boundary solve on z = 0 and P = 0 on the
 *     top and side faces (Sect. 2.2, three-step procedure);
 *   - Sect. 2.2: B_x = alpha P_y + P_xz, B_y = -alpha P_x + P_yz,
 *     B_z = -(P_xx + P_yy) by second-order finite differences;
 *   - eqs. (pressure) and (density) for p and rho, with the background
 *     atmosphere of Sect. 3 (piecewise temperature, ideal gas, hydrostatic).
 *
 * Discretisation: vertex-centred nodes x_i = i*hx, hx = Lx/(nx-1) (same in y
 * and z), array index i + nx*(j + ny*k) (x fastest, as in the flattened
 * offset of the Sect. 4 kernel listing, extended by k*nx*ny).
 *
 * Multigrid: V(nu1,nu2) cycles, red-black Gauss-Seidel smoothing (the paper
 * names Gauss-Jacobi; any convergent smoother reaches the same discrete
 * solution), full-weighting restriction, (bi/tri)linear prolongation,
 * re-discretised coarse operators, coarsest level solved by sweeping to
 * convergence.
 *
 * Parallelism: optional OpenMP over z-planes for the 3D loops.  Within one
 * colour every update is independent, and norms are summed per plane and
 * then serially, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, k, nx, ny) ((size_t)(i) + (size_t)(nx) * ((size_t)(j) + (size_t)(ny) * (size_t)(k)))

typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double alpha;
    int xi_kind; /* 0: xi = 0; 1: a exp(-kappa z); 2: (a + b sin(omega z)) exp(-kappa z) */
    double xi_a, xi_kappa, xi_b, xi_omega;
    double g, mu0, T_cor, z1, z2;
} orc_problem;

typedef struct {
    int cycles_2d, cycles_3d;
    double rel_res_2d, rel_res_3d;
    double conv_factor_3d;      /* geometric mean of the per-cycle residual ratios */
} orc_info;

/* ------------------------------------------------------------------------ */
/* Height profiles: xi(z) and its derivative (Sect. 3.2, xi_1 and xi_2        */
/* families); background atmosphere T_b, p_b, rho_b (Sect. 3).               */
/* ------------------------------------------------------------------------ */

double orc_xi(const orc_problem* p, double z) {
    switch (p->xi_kind) {
    case 1: return p->xi_a * exp(-p->xi_kappa * z);
    case 2: return (p->xi_a + p->xi_b * sin(p->xi_omega * z)) * exp(-p->xi_kappa * z);
    default: return 0.0;
    }
}

double orc_dxi(const orc_problem* p, double z) {
    switch (p->xi_kind) {
    case 1: return -p->xi_kappa * p->xi_a * exp(-p->xi_kappa * z);
    case 2:
        return (p->xi_b * p->xi_omega * cos(p->xi_omega * z) -
                p->xi_kappa * (p->xi_a + p->xi_b * sin(p->xi_omega * z))) * exp(-p->xi_kappa * z);
    default: return 0.0;
    }
}

/* T_b = 1 below z1, T_cor^((z - z1)/(z2 - z1)) between z1 and z2, T_cor above. */
double orc_Tb(const orc_problem* p, double z) {
    if (z <= p->z1) return 1.0;
    if (z <= p->z2) return pow(p->T_cor, (z - p->z1) / (p->z2 - p->z1));
    return p->T_cor;
}

/* Hydrostatic balance dp_b/dz = -g p_b / T_b with p_b(0) = 1, integrated in
 * closed form piece by piece: 1/T_b is constant or exponential in z. */
double orc_pb(const orc_problem* p, double z) {
    const double g = p->g, d = p->z2 - p->z1, lnT = log(p->T_cor);
    if (z <= p->z1) return exp(-g * z);
    const double p1 = exp(-g * p->z1);
    if (z <= p->z2) return p1 * exp(-g * d * (1.0 - pow(p->T_cor, -(z - p->z1) / d)) / lnT);
    const double p2 = p1 * exp(-g * d * (1.0 - 1.0 / p->T_cor) / lnT);
    return p2 * exp(-g * (z - p->z2) / p->T_cor);
}

double orc_rhob(const orc_problem* p, double z) { return orc_pb(p, z) / orc_Tb(p, z); }

/* ------------------------------------------------------------------------ */
/* One multigrid level of the 3D operator of eq. (scalar_pot):               */
/*   (A u)_ijk = cx_k (u_{i+1} + u_{i-1}) + cy_k (u_{j+1} + u_{j-1})         */
/*             + cz (u_{k+1} + u_{k-1}) + diag_k u_ijk                        */
/* with cx_k = (1 - xi(z_k))/hx^2, cy_k = (1 - xi(z_k))/hy^2, cz = 1/hz^2,    */
/* diag_k = -2 cx_k - 2 cy_k - 2 cz + alpha^2.                                */
/* The 2D operator of eq. (lower_bound) is the same with nz = 1, xi = 0,      */
/* no z terms and no alpha^2.                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    double* cx; /* per plane */
    double* cy;
    double* diag;
    double cz;
} orc_level;

static void level_init3d(orc_level* L, const orc_problem* p, int nx, int ny, int nz) {
    L->nx = nx; L->ny = ny; L->nz = nz;
    L->hx = p->Lx / (nx - 1);
    L->hy = p->Ly / (ny - 1);
    L->hz = p->Lz / (nz - 1);
    L->cz = 1.0 / (L->hz * L->hz);
    L->cx = (double*)malloc(sizeof(double) * nz);
    L->cy = (double*)malloc(sizeof(double) * nz);
    L->diag = (double*)malloc(sizeof(double) * nz);
    for (int k = 0; k < nz; ++k) {
        const double one_m_xi = 1.0 - orc_xi(p, k * L->hz);
        L->cx[k] = one_m_xi / (L->hx * L->hx);
        L->cy[k] = one_m_xi / (L->hy * L->hy);
        L->diag[k] = -2.0 * L->cx[k] - 2.0 * L->cy[k] - 2.0 * L->cz + p->alpha * p->alpha;
    }
}

static void level_init2d(orc_level* L, const orc_problem* p, int nx, int ny) {
    L->nx = nx; L->ny = ny; L->nz = 1;
    L->hx = p->Lx / (nx - 1);
    L->hy = p->Ly / (ny - 1);
    L->hz = 0.0;
    L->cz = 0.0;
    L->cx = (double*)malloc(sizeof(double));
    L->cy = (double*)malloc(sizeof(double));
    L->diag = (double*)malloc(sizeof(double));
    L->cx[0] = 1.0 / (L->hx * L->hx);
    L->cy[0] = 1.0 / (L->hy * L->hy);
    L->diag[0] = -2.0 * L->cx[0] - 2.0 * L->cy[0];
}

static void level_free(orc_level* L) { free(L->cx); free(L->cy); free(L->diag); }

static size_t level_size(const orc_level* L) { return (size_t)L->nx * L->ny * L->nz; }

/* r = f - A u at interior nodes, 0 on the boundary.  f may be NULL (zero). */
static void residual3d(const orc_level* L, const double* u, const double* f, double* r) {
    const int nx = L->nx, ny = L->ny, nz = L->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t c = IDX(i, j, k, nx, ny);
                if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) {
                    r[c] = 0.0;
                    continue;
                }
                const double Au = L->cx[k] * (u[c + 1] + u[c - 1]) +
                                  L->cy[k] * (u[c + nx] + u[c - nx]) +
                                  L->cz * (u[c + (size_t)nx * ny] + u[c - (size_t)nx * ny]) +
                                  L->diag[k] * u[c];
                r[c] = (f ? f[c] : 0.0) - Au;
            }
}

static void residual2d(const orc_level* L, const double* u, const double* f, double* r) {
    const int nx = L->nx, ny = L->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t c = IDX(i, j, 0, nx, ny);
            if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) { r[c] = 0.0; continue; }
            const double Au = L->cx[0] * (u[c + 1] + u[c - 1]) + L->cy[0] * (u[c + nx] + u[c - nx]) +
                              L->diag[0] * u[c];
            r[c] = (f ? f[c] : 0.0) - Au;
        }
}

/* One Gauss-Seidel pass over the nodes of one colour: solve row c of A u = f
 * for u_c with the current neighbour values. */
static void rbgs3d_colour(const orc_level* L, double* u, const double* f, int colour) {
    const int nx = L->nx, ny = L->ny, nz = L->nz;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                if (((i + j + k) & 1) != colour) continue;
                const size_t c = IDX(i, j, k, nx, ny);
                const double off = L->cx[k] * (u[c + 1] + u[c - 1]) +
                                   L->cy[k] * (u[c + nx] + u[c - nx]) +
                                   L->cz * (u[c + (size_t)nx * ny] + u[c - (size_t)nx * ny]);
                u[c] = ((f ? f[c] : 0.0) - off) / L->diag[k];
            }
}

static void rbgs2d_colour(const orc_level* L, double* u, const double* f, int colour) {
    const int nx = L->nx, ny = L->ny;
    for (int j = 1; j < ny - 1; ++j)
        for (int i = 1; i < nx - 1; ++i) {
            if (((i + j) & 1) != colour) continue;
            const size_t c = IDX(i, j, 0, nx, ny);
            const double off = L->cx[0] * (u[c + 1] + u[c - 1]) + L->cy[0] * (u[c + nx] + u[c - nx]);
            u[c] = ((f ? f[c] : 0.0) - off) / L->diag[0];
        }
}

/* A red-black sweep: colour 0 ((i+j+k) even) first, then colour 1. */
static void rbgs3d(const orc_level* L, double* u, const double* f) {
    rbgs3d_colour(L, u, f, 0);
    rbgs3d_colour(L, u, f, 1);
}

static void rbgs2d(const orc_level* L, double* u, const double* f) {
    rbgs2d_colour(L, u, f, 0);
    rbgs2d_colour(L, u, f, 1);
}

/* Zebra z-line Gauss-Seidel, the line-relaxation form of the Sect. 4
 * smoother for strong vertical coupling (xi(z) near 1, or h_z < h_x, where
 * [1 - xi] (P_xx + P_yy) is small next to P_zz).  The columns (i, j) are
 * coloured by the parity of i + j.  For every column of the colour, the
 * nz - 2 interior rows of A u = f along the column are solved exactly for
 * u(i, j, 1 .. nz-2), with the neighbouring columns and the Dirichlet values
 * u(i, j, 0), u(i, j, nz-1) held at their current values:
 *   cz u[k-1] + diag[k] u[k] + cz u[k+1] = f[k] - cx[k] (u_E + u_W) - cy[k] (u_N + u_S).
 * The tridiagonal system is solved by Gaussian elimination without pivoting
 * (the Thomas algorithm); -A is symmetric positive definite, so no pivot
 * vanishes. */
static void zline3d_colour(const orc_level* L, double* u, const double* f, int colour) {
    const int nx = L->nx, ny = L->ny, nz = L->nz, m = nz - 2;
    const size_t plane = (size_t)nx * ny;
    if (m < 1) return;
#pragma omp parallel
    {
        double* sup = (double*)malloc(sizeof(double) * m);   /* eliminated super-diagonal */
        double* rhs = (double*)malloc(sizeof(double) * m);   /* eliminated right-hand side */
#pragma omp for schedule(static)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                if (((i + j) & 1) != colour) continue;
                for (int t = 0; t < m; ++t) {
                    const int k = t + 1;
                    const size_t c = IDX(i, j, k, nx, ny);
                    double b = (f ? f[c] : 0.0) - L->cx[k] * (u[c + 1] + u[c - 1]) - L->cy[k] * (u[c + nx] + u[c - nx]);
                    if (k == 1) b -= L->cz * u[c - plane];
                    if (k == nz - 2) b -= L->cz * u[c + plane];
                    const double pivot = L->diag[k] - (t > 0 ? L->cz * sup[t - 1] : 0.0);
                    sup[t] = L->cz / pivot;
                    rhs[t] = (b - (t > 0 ? L->cz * rhs[t - 1] : 0.0)) / pivot;
                }
                for (int t = m - 1; t >= 0; --t) {
                    const size_t c = IDX(i, j, t + 1, nx, ny);
                    u[c] = rhs[t] - (t < m - 1 ? sup[t] * u[c + plane] : 0.0);
                }
            }
        free(sup);
        free(rhs);
    }
}

/* A zebra sweep: columns with i + j even first, then odd. */
static void zline3d(const orc_level* L, double* u, const double* f) {
    zline3d_colour(L, u, f, 0);
    zline3d_colour(L, u, f, 1);
}

/* Full weighting: tensor product of the 1D weights (1/4, 1/2, 1/4) around
 * the coincident fine node; coarse boundary nodes are set to 0. */
static void restrict3d(const orc_level* F, const double* rf, const orc_level* C, double* fc) {
    static const double w[3] = {0.25, 0.5, 0.25};
    const int nxc = C->nx, nyc = C->ny, nzc = C->nz, nx = F->nx, ny = F->ny;
#pragma omp parallel for schedule(static)
    for (int K = 0; K < nzc; ++K)
        for (int J = 0; J < nyc; ++J)
            for (int I = 0; I < nxc; ++I) {
                const size_t c = IDX(I, J, K, nxc, nyc);
                if (I == 0 || J == 0 || K == 0 || I == nxc - 1 || J == nyc - 1 || K == nzc - 1) {
                    fc[c] = 0.0;
                    continue;
                }
                double s = 0.0;
                for (int c3 = -1; c3 <= 1; ++c3)
                    for (int b = -1; b <= 1; ++b)
                        for (int a = -1; a <= 1; ++a)
                            s += w[a + 1] * w[b + 1] * w[c3 + 1] *
                                 rf[IDX(2 * I + a, 2 * J + b, 2 * K + c3, nx, ny)];
                fc[c] = s;
            }
}

static void restrict2d(const orc_level* F, const double* rf, const orc_level* C, double* fc) {
    static const double w[3] = {0.25, 0.5, 0.25};
    const int nxc = C->nx, nyc = C->ny, nx = F->nx, ny = F->ny;
    for (int J = 0; J < nyc; ++J)
        for (int I = 0; I < nxc; ++I) {
            const size_t c = IDX(I, J, 0, nxc, nyc);
            if (I == 0 || J == 0 || I == nxc - 1 || J == nyc - 1) { fc[c] = 0.0; continue; }
            double s = 0.0;
            for (int b = -1; b <= 1; ++b)
                for (int a = -1; a <= 1; ++a)
                    s += w[a + 1] * w[b + 1] * rf[IDX(2 * I + a, 2 * J + b, 0, nx, ny)];
            fc[c] = s;
        }
}

/* Linear interpolation along one axis: even fine index -> coarse node i/2
 * with weight 1; odd -> the two coarse neighbours with weight 1/2. */
static double lin_weight(int i, int I) {
    if ((i & 1) == 0) return (I * 2 == i) ? 1.0 : 0.0;
    return (I * 2 == i - 1 || I * 2 == i + 1) ? 0.5 : 0.0;
}

/* u_f += I e_c at fine interior nodes (trilinear interpolation). */
static void prolong_add3d(const orc_level* C, const double* ec, const orc_level* F, double* uf) {
    const int nx = F->nx, ny = F->ny, nz = F->nz, nxc = C->nx, nyc = C->ny;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                double s = 0.0;
                for (int K = (k - 1) / 2; K <= (k + 1) / 2; ++K)
                    for (int J = (j - 1) / 2; J <= (j + 1) / 2; ++J)
                        for (int I = (i - 1) / 2; I <= (i + 1) / 2; ++I)
                            s += lin_weight(i, I) * lin_weight(j, J) * lin_weight(k, K) *
                                 ec[IDX(I, J, K, nxc, nyc)];
                uf[IDX(i, j, k, nx, ny)] += s;
            }
}

static void prolong_add2d(const orc_level* C, const double* ec, const orc_level* F, double* uf) {
    const int nx = F->nx, ny = F->ny, nxc = C->nx, nyc = C->ny;
    for (int j = 1; j < ny - 1; ++j)
        for (int i = 1; i < nx - 1; ++i) {
            double s = 0.0;
            for (int J = (j - 1) / 2; J <= (j + 1) / 2; ++J)
                for (int I = (i - 1) / 2; I <= (i + 1) / 2; ++I)
                    s += lin_weight(i, I) * lin_weight(j, J) * ec[IDX(I, J, 0, nxc, nyc)];
            uf[IDX(i, j, 0, nx, ny)] += s;
        }
}

/* Euclidean norm over the array (boundary entries of a residual are 0).
 * Summed per plane, then over planes in order: independent of threads. */
static double norm2(const double* v, int nx, int ny, int nz) {
    double* part = (double*)malloc(sizeof(double) * nz);
    const size_t plane = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double s = 0.0;
        for (size_t c = 0; c < plane; ++c) s += v[k * plane + c] * v[k * plane + c];
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += part[k];
    free(part);
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Multigrid hierarchy and V-cycle                                           */
/* ------------------------------------------------------------------------ */

#define ORC_MAX_LEVELS 16

typedef struct {
    int nlev;
    int dim; /* 2 or 3 */
    orc_level L[ORC_MAX_LEVELS];
    double* u[ORC_MAX_LEVELS]; /* level 0's u is the caller's array */
    double* f[ORC_MAX_LEVELS];
    double* r[ORC_MAX_LEVELS];
    int smoother; /* 0: red-black point Gauss-Seidel; 1: zebra z-line Gauss-Seidel (3D levels) */
    int exact_level; /* level whose system a V-cycle solves to rounding instead of descending (-1: none) */
} orc_mg;

static int coarsenable(int n) { return n >= 5 && ((n - 1) % 2) == 0; }

static void mg_build(orc_mg* mg, const orc_problem* p, int dim) {
    int nx = p->nx, ny = p->ny, nz = (dim == 3) ? p->nz : 1;
    mg->dim = dim;
    mg->nlev = 0;
    mg->smoother = 0;
    mg->exact_level = -1;
    for (;;) {
        orc_level* L = &mg->L[mg->nlev];
        if (dim == 3) level_init3d(L, p, nx, ny, nz); else level_init2d(L, p, nx, ny);
        const size_t n = level_size(L);
        mg->u[mg->nlev] = (double*)calloc(n, sizeof(double));
        mg->f[mg->nlev] = (double*)calloc(n, sizeof(double));
        mg->r[mg->nlev] = (double*)calloc(n, sizeof(double));
        mg->nlev++;
        const int can = coarsenable(nx) && coarsenable(ny) && (dim == 2 || coarsenable(nz));
        if (!can || mg->nlev == ORC_MAX_LEVELS) break;
        nx = (nx - 1) / 2 + 1; ny = (ny - 1) / 2 + 1;
        if (dim == 3) nz = (nz - 1) / 2 + 1;
    }
}

static void mg_free(orc_mg* mg) {
    for (int l = 0; l < mg->nlev; ++l) {
        level_free(&mg->L[l]);
        free(mg->u[l]); free(mg->f[l]); free(mg->r[l]);
    }
}

static void mg_residual(const orc_mg* mg, int l, const double* u, const double* f, double* r) {
    if (mg->dim == 3) residual3d(&mg->L[l], u, f, r); else residual2d(&mg->L[l], u, f, r);
}

static void mg_smooth(const orc_mg* mg, int l, double* u, const double* f) {
    if (mg->dim == 3) {
        if (mg->smoother == 1) zline3d(&mg->L[l], u, f); else rbgs3d(&mg->L[l], u, f);
    } else {
        rbgs2d(&mg->L[l], u, f);
    }
}

static double mg_norm(const orc_mg* mg, int l, const double* v) {
    return norm2(v, mg->L[l].nx, mg->L[l].ny, mg->L[l].nz);
}

/* Coarsest level: sweep until the residual falls 1e-14 below the right-hand
 * side (or a sweep cap). */
static void coarse_solve(orc_mg* mg, int l, double* u, const double* f) {
    const double fn = mg_norm(mg, l, f);
    for (int it = 0; it < 100000; ++it) {
        mg_smooth(mg, l, u, f);
        if ((it & 7) == 7) {
            mg_residual(mg, l, u, f, mg->r[l]);
            if (mg_norm(mg, l, mg->r[l]) <= 1e-14 * fn) break;
        }
    }
}

static void vcycle(orc_mg* mg, int l, double* u, const double* f, int nu1, int nu2);

/* Coarse-grid correction solved exactly: the level's system A u = f (zero
 * boundary values) iterated to rounding by V-cycles over the coarser levels,
 * until the residual stops falling or is 1e-15 of ||f||.  Any method that
 * reaches the exact solution of the coarse system serves here. */
static void exact_solve(orc_mg* mg, int l, double* u, const double* f, int nu1, int nu2) {
    const int saved = mg->exact_level;
    mg->exact_level = -1;
    const double fn = mg_norm(mg, l, f);
    double prev = INFINITY;
    for (int it = 0; it < 200; ++it) {
        mg_residual(mg, l, u, f, mg->r[l]);
        const double rn = mg_norm(mg, l, mg->r[l]);
        if (rn <= 1e-15 * fn || rn > 0.5 * prev) break;
        prev = rn;
        vcycle(mg, l, u, f, nu1, nu2);
    }
    mg->exact_level = saved;
}

static void vcycle(orc_mg* mg, int l, double* u, const double* f, int nu1, int nu2) {
    if (l == mg->nlev - 1) { coarse_solve(mg, l, u, f); return; }
    if (l == mg->exact_level) { exact_solve(mg, l, u, f, nu1, nu2); return; }
    for (int s = 0; s < nu1; ++s) mg_smooth(mg, l, u, f);
    mg_residual(mg, l, u, f, mg->r[l]);
    if (mg->dim == 3) restrict3d(&mg->L[l], mg->r[l], &mg->L[l + 1], mg->f[l + 1]);
    else restrict2d(&mg->L[l], mg->r[l], &mg->L[l + 1], mg->f[l + 1]);
    memset(mg->u[l + 1], 0, sizeof(double) * level_size(&mg->L[l + 1]));
    vcycle(mg, l + 1, mg->u[l + 1], mg->f[l + 1], nu1, nu2);
    if (mg->dim == 3) prolong_add3d(&mg->L[l + 1], mg->u[l + 1], &mg->L[l], u);
    else prolong_add2d(&mg->L[l + 1], mg->u[l + 1], &mg->L[l], u);
    for (int s = 0; s < nu2; ++s) mg_smooth(mg, l, u, f);
}

/* Solve A u = f on the finest level of mg by V-cycles, starting from u (whose
 * boundary entries carry the Dirichlet data).  Stops when
 * ||f - A u|| / ||b|| < tol, b being the residual of u with its interior set
 * to zero (the right-hand side after the Dirichlet data is lifted).
 * history (length max_cycles + 1, may be NULL) receives the relative
 * residual after each cycle, entry 0 the start.  Returns the cycle count. */
static int mg_solve(orc_mg* mg, double* u, const double* f, double tol, int max_cycles, int nu1, int nu2,
                    double* rel_out, double* history, double* conv_out) {
    const orc_level* L = &mg->L[0];
    const size_t n = level_size(L);
    double* lift = (double*)malloc(sizeof(double) * n);
    memcpy(lift, u, sizeof(double) * n);
    for (int k = (mg->dim == 3 ? 1 : 0); k < (mg->dim == 3 ? L->nz - 1 : 1); ++k)
        for (int j = 1; j < L->ny - 1; ++j)
            for (int i = 1; i < L->nx - 1; ++i) lift[IDX(i, j, k, L->nx, L->ny)] = 0.0;
    mg_residual(mg, 0, lift, f, mg->r[0]);
    const double bnorm = mg_norm(mg, 0, mg->r[0]);
    free(lift);
    mg_residual(mg, 0, u, f, mg->r[0]);
    double rn = mg_norm(mg, 0, mg->r[0]);
    double rel = (bnorm > 0.0) ? rn / bnorm : 0.0;
    const double rel0 = rel;
    if (history) history[0] = rel;
    int cyc = 0;
    while (rel >= tol && cyc < max_cycles && bnorm > 0.0) {
        vcycle(mg, 0, u, f, nu1, nu2);
        mg_residual(mg, 0, u, f, mg->r[0]);
        rn = mg_norm(mg, 0, mg->r[0]);
        rel = rn / bnorm;
        ++cyc;
        if (history) history[cyc] = rel;
    }
    if (rel_out) *rel_out = rel;
    if (conv_out) *conv_out = (cyc > 0 && rel0 > 0.0 && rel > 0.0) ? pow(rel / rel0, 1.0 / cyc) : 0.0;
    return cyc;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (called through ctypes from the tests)             */
/* ------------------------------------------------------------------------ */

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Per-plane coefficients of the 3D operator on the finest level. */
void orc_coeffs(const orc_problem* p, double* cx, double* cy, double* cz, double* diag) {
    orc_level L;
    level_init3d(&L, p, p->nx, p->ny, p->nz);
    memcpy(cx, L.cx, sizeof(double) * p->nz);
    memcpy(cy, L.cy, sizeof(double) * p->nz);
    memcpy(diag, L.diag, sizeof(double) * p->nz);
    *cz = L.cz;
    level_free(&L);
}

/* Single operations on one 3D grid of size nx*ny*nz of problem p (the grid
 * may be a coarse level: spacings come from p's lengths and these counts). */
static orc_problem with_size(const orc_problem* p, int nx, int ny, int nz) {
    orc_problem q = *p;
    q.nx = nx; q.ny = ny; q.nz = nz;
    return q;
}

void orc_residual3d(const orc_problem* p, int nx, int ny, int nz, const double* u, const double* f, double* r) {
    orc_problem q = with_size(p, nx, ny, nz);
    orc_level L;
    level_init3d(&L, &q, nx, ny, nz);
    residual3d(&L, u, f, r);
    level_free(&L);
}

void orc_rbgs3d(const orc_problem* p, int nx, int ny, int nz, double* u, const double* f, int sweeps) {
    orc_problem q = with_size(p, nx, ny, nz);
    orc_level L;
    level_init3d(&L, &q, nx, ny, nz);
    for (int s = 0; s < sweeps; ++s) rbgs3d(&L, u, f);
    level_free(&L);
}

void orc_rbgs3d_colour(const orc_problem* p, int nx, int ny, int nz, double* u, const double* f, int colour) {
    orc_problem q = with_size(p, nx, ny, nz);
    orc_level L;
    level_init3d(&L, &q, nx, ny, nz);
    rbgs3d_colour(&L, u, f, colour);
    level_free(&L);
}

void orc_zline3d(const orc_problem* p, int nx, int ny, int nz, double* u, const double* f, int sweeps) {
    orc_problem q = with_size(p, nx, ny, nz);
    orc_level L;
    level_init3d(&L, &q, nx, ny, nz);
    for (int s = 0; s < sweeps; ++s) zline3d(&L, u, f);
    level_free(&L);
}

void orc_zline3d_colour(const orc_problem* p, int nx, int ny, int nz, double* u, const double* f, int colour) {
    orc_problem q = with_size(p, nx, ny, nz);
    orc_level L;
    level_init3d(&L, &q, nx, ny, nz);
    zline3d_colour(&L, u, f, colour);
    level_free(&L);
}

void orc_residual2d(const orc_problem* p, int nx, int ny, const double* u, const double* f, double* r) {
    orc_problem q = with_size(p, nx, ny, 1);
    orc_level L;
    level_init2d(&L, &q, nx, ny);
    residual2d(&L, u, f, r);
    level_free(&L);
}

void orc_rbgs2d(const orc_problem* p, int nx, int ny, double* u, const double* f, int sweeps) {
    orc_problem q = with_size(p, nx, ny, 1);
    orc_level L;
    level_init2d(&L, &q, nx, ny);
    for (int s = 0; s < sweeps; ++s) rbgs2d(&L, u, f);
    level_free(&L);
}

/* Restriction / prolongation between a fine grid (nx,ny,nz) and its coarse
 * grid ((n-1)/2+1 per axis).  Pass nz = 1 for the 2D operators. */
void orc_restrict(int nx, int ny, int nz, const double* rf, double* fc) {
    orc_level F = {nx, ny, nz, 0, 0, 0, 0, 0, 0, 0};
    orc_level C = {(nx - 1) / 2 + 1, (ny - 1) / 2 + 1, nz == 1 ? 1 : (nz - 1) / 2 + 1, 0, 0, 0, 0, 0, 0, 0};
    if (nz == 1) restrict2d(&F, rf, &C, fc); else restrict3d(&F, rf, &C, fc);
}

void orc_prolong_add(int nx, int ny, int nz, const double* ec, double* uf) {
    orc_level F = {nx, ny, nz, 0, 0, 0, 0, 0, 0, 0};
    orc_level C = {(nx - 1) / 2 + 1, (ny - 1) / 2 + 1, nz == 1 ? 1 : (nz - 1) / 2 + 1, 0, 0, 0, 0, 0, 0, 0};
    if (nz == 1) prolong_add2d(&C, ec, &F, uf); else prolong_add3d(&C, ec, &F, uf);
}

/* Lower-boundary solve, eq. (lower_bound): P0_xx + P0_yy = -bz on the
 * interior of the nx*ny plane, P0 = 0 on its edges.  P0 is overwritten (its
 * interior is the initial guess; zero it for the paper's start). */
int orc_solve2d(const orc_problem* p, const double* bz, double* P0, double tol, int max_cycles, int nu1, int nu2,
                double* rel_out, double* history) {
    orc_mg mg;
    mg_build(&mg, p, 2);
    const int nx = p->nx, ny = p->ny;
    double* f = (double*)calloc((size_t)nx * ny, sizeof(double));
    for (int j = 1; j < ny - 1; ++j)
        for (int i = 1; i < nx - 1; ++i) f[IDX(i, j, 0, nx, ny)] = -bz[IDX(i, j, 0, nx, ny)];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) P0[IDX(i, j, 0, nx, ny)] = 0.0;
    const int cyc = mg_solve(&mg, P0, f, tol, max_cycles, nu1, nu2, rel_out, history, NULL);
    free(f);
    mg_free(&mg);
    return cyc;
}

/* Interior solve, eq. (scalar_pot), with right-hand side f (NULL = 0).  P's
 * boundary entries are the Dirichlet data (plane k = 0 from the lower
 * boundary solve, 0 elsewhere for the paper's problem); its interior is the
 * initial guess. */
int orc_solve3d_s(const orc_problem* p, double* P, const double* f, double tol, int max_cycles, int nu1, int nu2,
                  int smoother, double* rel_out, double* history, double* conv_out) {
    orc_mg mg;
    mg_build(&mg, p, 3);
    mg.smoother = smoother;
    const int cyc = mg_solve(&mg, P, f, tol, max_cycles, nu1, nu2, rel_out, history, conv_out);
    mg_free(&mg);
    return cyc;
}

int orc_solve3d(const orc_problem* p, double* P, const double* f, double tol, int max_cycles, int nu1, int nu2,
                double* rel_out, double* history, double* conv_out) {
    return orc_solve3d_s(p, P, f, tol, max_cycles, nu1, nu2, 0, rel_out, history, conv_out);
}

int orc_num_levels(const orc_problem* p, int dim) {
    orc_mg mg;
    mg_build(&mg, p, dim);
    const int n = mg.nlev;
    mg_free(&mg);
    return n;
}

/* The numerical procedure of Sect. 2.2: (1) P = 0 everywhere; (2) multigrid
 * on z = 0 for eq. (lower_bound); (3) multigrid in the interior for
 * eq. (scalar_pot) with the plane k = 0 from step 2 and P = 0 on the top and
 * sides.  P has nx*ny*nz entries. */
int orc_solve_s(const orc_problem* p, const double* bz, double* P, double tol2d, double tol3d, int max_cycles,
                int nu1, int nu2, int smoother, orc_info* info) {
    const size_t plane = (size_t)p->nx * p->ny;
    memset(P, 0, sizeof(double) * plane * p->nz);
    double rel2 = 0.0, rel3 = 0.0, conv = 0.0;
    const int c2 = orc_solve2d(p, bz, P, tol2d, max_cycles, nu1, nu2, &rel2, NULL);
    const int c3 = orc_solve3d_s(p, P, NULL, tol3d, max_cycles, nu1, nu2, smoother, &rel3, NULL, &conv);
    if (info) {
        info->cycles_2d = c2; info->cycles_3d = c3;
        info->rel_res_2d = rel2; info->rel_res_3d = rel3;
        info->conv_factor_3d = conv;
    }
    return (rel2 < tol2d && rel3 < tol3d) ? 0 : 1;
}

int orc_solve(const orc_problem* p, const double* bz, double* P, double tol2d, double tol3d, int max_cycles,
              int nu1, int nu2, orc_info* info) {
    return orc_solve_s(p, bz, P, tol2d, tol3d, max_cycles, nu1, nu2, 0, info);
}

/* ------------------------------------------------------------------------ */
/* Finite differences (Sect. 2.2): central inside, second-order one-sided at */
/* the first and last node of an axis.                                       */
/* ------------------------------------------------------------------------ */

/* d/dx_axis of f at node (i,j,k) along axis a (0: x, 1: y, 2: z). */
static double d1(const double* f, int nx, int ny, int nz, int i, int j, int k, int a, double h) {
    const int n = (a == 0) ? nx : (a == 1) ? ny : nz;
    const int t = (a == 0) ? i : (a == 1) ? j : k;
    const size_t s = (a == 0) ? 1 : (a == 1) ? (size_t)nx : (size_t)nx * ny;
    const size_t c = IDX(i, j, k, nx, ny);
    if (t == 0) return (-3.0 * f[c] + 4.0 * f[c + s] - f[c + 2 * s]) / (2.0 * h);
    if (t == n - 1) return (3.0 * f[c] - 4.0 * f[c - s] + f[c - 2 * s]) / (2.0 * h);
    return (f[c + s] - f[c - s]) / (2.0 * h);
}

/* d^2/dx_axis^2 (compact three-point inside, four-point one-sided at ends). */
static double d2(const double* f, int nx, int ny, int nz, int i, int j, int k, int a, double h) {
    const int n = (a == 0) ? nx : (a == 1) ? ny : nz;
    const int t = (a == 0) ? i : (a == 1) ? j : k;
    const size_t s = (a == 0) ? 1 : (a == 1) ? (size_t)nx : (size_t)nx * ny;
    const size_t c = IDX(i, j, k, nx, ny);
    if (t == 0) return (2.0 * f[c] - 5.0 * f[c + s] + 4.0 * f[c + 2 * s] - f[c + 3 * s]) / (h * h);
    if (t == n - 1) return (2.0 * f[c] - 5.0 * f[c - s] + 4.0 * f[c - 2 * s] - f[c - 3 * s]) / (h * h);
    return (f[c + s] - 2.0 * f[c] + f[c - s]) / (h * h);
}

/* Apply d1 along axis a to the whole array. */
static void d1_all(const double* f, double* out, int nx, int ny, int nz, int a, double h) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) out[IDX(i, j, k, nx, ny)] = d1(f, nx, ny, nz, i, j, k, a, h);
}

/* B, p and rho from P.  bz_mode 0: B_z = -(d2_x + d2_y) P (the compact
 * operator of the lower-boundary solve); bz_mode 1: B_z = -(d1_x d1_x + d1_y
 * d1_y) P, which makes the central-difference divergence of B vanish to
 * rounding.  Any output pointer may be NULL; Bz is computed internally when
 * rho is wanted. */
void orc_fields(const orc_problem* p, const double* P, double* Bx, double* By, double* Bz, double* pr,
                double* rho, int bz_mode) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double hx = p->Lx / (nx - 1), hy = p->Ly / (ny - 1), hz = p->Lz / (nz - 1);
    const size_t n = (size_t)nx * ny * nz;
    double* Pz = (double*)malloc(sizeof(double) * n);   /* dP/dz */
    double* Px = (double*)malloc(sizeof(double) * n);   /* dP/dx */
    double* Py = (double*)malloc(sizeof(double) * n);   /* dP/dy */
    double* bx = (double*)malloc(sizeof(double) * n);
    double* by = (double*)malloc(sizeof(double) * n);
    double* bz = (double*)malloc(sizeof(double) * n);
    d1_all(P, Pz, nx, ny, nz, 2, hz);
    d1_all(P, Px, nx, ny, nz, 0, hx);
    d1_all(P, Py, nx, ny, nz, 1, hy);
    double* Pxx = NULL; double* Pyy = NULL;
    if (bz_mode == 1) {
        Pxx = (double*)malloc(sizeof(double) * n);
        Pyy = (double*)malloc(sizeof(double) * n);
        d1_all(Px, Pxx, nx, ny, nz, 0, hx);
        d1_all(Py, Pyy, nx, ny, nz, 1, hy);
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t c = IDX(i, j, k, nx, ny);
                bx[c] = p->alpha * Py[c] + d1(Pz, nx, ny, nz, i, j, k, 0, hx);
                by[c] = -p->alpha * Px[c] + d1(Pz, nx, ny, nz, i, j, k, 1, hy);
                if (bz_mode == 1) bz[c] = -(Pxx[c] + Pyy[c]);
                else bz[c] = -(d2(P, nx, ny, nz, i, j, k, 0, hx) + d2(P, nx, ny, nz, i, j, k, 1, hy));
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        const double z = k * hz;
        const double xi = orc_xi(p, z), dxi = orc_dxi(p, z), pb = orc_pb(p, z), rb = orc_rhob(p, z);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t c = IDX(i, j, k, nx, ny);
                const double B2 = bz[c] * bz[c] / (2.0 * p->mu0);
                if (pr) pr[c] = pb - xi * B2;
                if (rho) {
                    const double BgradBz = bx[c] * d1(bz, nx, ny, nz, i, j, k, 0, hx) +
                                           by[c] * d1(bz, nx, ny, nz, i, j, k, 1, hy) +
                                           bz[c] * d1(bz, nx, ny, nz, i, j, k, 2, hz);
                    rho[c] = rb + (dxi * B2 + xi * BgradBz / p->mu0) / p->g;
                }
            }
    }
    if (Bx) memcpy(Bx, bx, sizeof(double) * n);
    if (By) memcpy(By, by, sizeof(double) * n);
    if (Bz) memcpy(Bz, bz, sizeof(double) * n);
    free(Pz); free(Px); free(Py); free(bx); free(by); free(bz);
    free(Pxx); free(Pyy);
}

/* Background profiles and xi on the nz node heights z_k = k Lz/(nz-1). */
void orc_profiles(const orc_problem* p, double* xi, double* dxi, double* pb, double* rhob, double* Tb) {
    const double hz = p->Lz / (p->nz - 1);
    for (int k = 0; k < p->nz; ++k) {
        const double z = k * hz;
        if (xi) xi[k] = orc_xi(p, z);
        if (dxi) dxi[k] = orc_dxi(p, z);
        if (pb) pb[k] = orc_pb(p, z);
        if (rhob) rhob[k] = orc_rhob(p, z);
        if (Tb) Tb[k] = orc_Tb(p, z);
    }
}

/* One V(nu1,nu2)-cycle for A u = f on the grid of u (dim 3: nx*ny*nz,
 * dim 2: nx*ny), from that grid down to the coarsest level, or, with
 * exact_level >= 1, down to that level, whose coarse-grid system is solved
 * to rounding.  u is updated in place; its boundary entries are the
 * Dirichlet data. */
void orc_vcycle_x(const orc_problem* p, int dim, int nx, int ny, int nz, double* u, const double* f, int nu1,
                  int nu2, int smoother, int exact_level) {
    orc_problem q = with_size(p, nx, ny, dim == 3 ? nz : 1);
    orc_mg mg;
    mg_build(&mg, &q, dim);
    mg.smoother = smoother;
    mg.exact_level = exact_level >= 1 ? exact_level : -1;
    const size_t n = level_size(&mg.L[0]);
    double* fz = NULL;
    if (!f) fz = (double*)calloc(n, sizeof(double));
    vcycle(&mg, 0, u, f ? f : fz, nu1, nu2);
    free(fz);
    mg_free(&mg);
}

void orc_vcycle_s(const orc_problem* p, int dim, int nx, int ny, int nz, double* u, const double* f, int nu1,
                  int nu2, int smoother) {
    orc_vcycle_x(p, dim, nx, ny, nz, u, f, nu1, nu2, smoother, -1);
}

void orc_vcycle(const orc_problem* p, int dim, int nx, int ny, int nz, double* u, const double* f, int nu1,
                int nu2) {
    orc_vcycle_s(p, dim, nx, ny, nz, u, f, nu1, nu2, 0);
}

/* ------------------------------------------------------------------------ */
/* Post-processing for the paper's figure quantities (Sect. 3): current     */
/* density and magnetic field lines.                                         */
/* ------------------------------------------------------------------------ */

/* j = curl B / mu0 with the difference operators of the field recovery
 * (central inside, second-order one-sided at the first and last node of an
 * axis), and the magnitudes |j|, |B|.  Any output may be NULL. */
void orc_current(const orc_problem* p, const double* Bx, const double* By, const double* Bz, double* jx, double* jy,
                 double* jz, double* jmag, double* bmag) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double hx = p->Lx / (nx - 1), hy = p->Ly / (ny - 1), hz = p->Lz / (nz - 1);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t c = IDX(i, j, k, nx, ny);
                const double cx = (d1(Bz, nx, ny, nz, i, j, k, 1, hy) - d1(By, nx, ny, nz, i, j, k, 2, hz)) / p->mu0;
                const double cy = (d1(Bx, nx, ny, nz, i, j, k, 2, hz) - d1(Bz, nx, ny, nz, i, j, k, 0, hx)) / p->mu0;
                const double cz = (d1(By, nx, ny, nz, i, j, k, 0, hx) - d1(Bx, nx, ny, nz, i, j, k, 1, hy)) / p->mu0;
                if (jx) jx[c] = cx;
                if (jy) jy[c] = cy;
                if (jz) jz[c] = cz;
                if (jmag) jmag[c] = sqrt(cx * cx + cy * cy + cz * cz);
                if (bmag) bmag[c] = sqrt(Bx[c] * Bx[c] + By[c] * By[c] + Bz[c] * Bz[c]);
            }
}

/* Unit field direction dir * B/|B| at the point r of the box [0,Lx]x[0,Ly]x[0,Lz]
 * (node (i,j,k) at (i hx, j hy, k hz)), B interpolated trilinearly from the
 * eight nodes of the cell holding r (the last cell for points on an upper
 * face), first along x, then y, then z.  Returns 0 when r lies outside the
 * closed box or |B| vanishes there. */
static int trace_dir(const orc_problem* p, const double* B[3], double dir, const double r[3], double v[3]) {
    const int n[3] = {p->nx, p->ny, p->nz};
    const double L[3] = {p->Lx, p->Ly, p->Lz};
    int c[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        if (!(r[a] >= 0.0 && r[a] <= L[a])) return 0;
        const double h = L[a] / (n[a] - 1);
        const double s = r[a] / h;
        int i = (int)floor(s);
        if (i > n[a] - 2) i = n[a] - 2;
        if (i < 0) i = 0;
        c[a] = i;
        f[a] = s - i;
    }
    const int nx = p->nx, ny = p->ny;
    double b[3];
    for (int q = 0; q < 3; ++q) {
        const double* F = B[q];
        double e[2][2];
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy) {
                const double f0 = F[IDX(c[0], c[1] + dy, c[2] + dz, nx, ny)];
                const double f1 = F[IDX(c[0] + 1, c[1] + dy, c[2] + dz, nx, ny)];
                e[dz][dy] = f0 * (1.0 - f[0]) + f1 * f[0];
            }
        const double e0 = e[0][0] * (1.0 - f[1]) + e[0][1] * f[1];
        const double e1 = e[1][0] * (1.0 - f[1]) + e[1][1] * f[1];
        b[q] = e0 * (1.0 - f[2]) + e1 * f[2];
    }
    const double m = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    if (!(m > 0.0)) return 0;
    for (int q = 0; q < 3; ++q) v[q] = dir * b[q] / m;
    return 1;
}

/* Field lines: for each of the n seeds (x, y, z), classical fourth-order
 * Runge-Kutta steps of length ds along dr/ds = dir B/|B| (dir = +1 along B,
 * -1 against it), at most max_steps of them.  A step is taken only when all
 * four stage points and its end point lie in the closed box and |B| does not
 * vanish at the stage points; otherwise the line ends.  points holds
 * n x (max_steps + 1) x 3 coordinates, the seed first; lengths[q] is the
 * number of points of line q (0 for a seed outside the box). */
void orc_trace(const orc_problem* p, const double* Bx, const double* By, const double* Bz, const double* seeds, int n,
               double ds, int max_steps, double dir, double* points, int* lengths) {
    const double* B[3] = {Bx, By, Bz};
    const double L[3] = {p->Lx, p->Ly, p->Lz};
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < n; ++q) {
        double r[3] = {seeds[3 * q], seeds[3 * q + 1], seeds[3 * q + 2]};
        double* out = points + (size_t)q * (max_steps + 1) * 3;
        int inside = 1;
        for (int a = 0; a < 3; ++a) inside = inside && r[a] >= 0.0 && r[a] <= L[a];
        if (!inside) { lengths[q] = 0; continue; }
        out[0] = r[0]; out[1] = r[1]; out[2] = r[2];
        int len = 1;
        const double hs = 0.5 * ds, s6 = ds / 6.0;
        for (int step = 0; step < max_steps; ++step) {
            double k1[3], k2[3], k3[3], k4[3], t[3], e[3];
            if (!trace_dir(p, B, dir, r, k1)) break;
            for (int a = 0; a < 3; ++a) t[a] = r[a] + hs * k1[a];
            if (!trace_dir(p, B, dir, t, k2)) break;
            for (int a = 0; a < 3; ++a) t[a] = r[a] + hs * k2[a];
            if (!trace_dir(p, B, dir, t, k3)) break;
            for (int a = 0; a < 3; ++a) t[a] = r[a] + ds * k3[a];
            if (!trace_dir(p, B, dir, t, k4)) break;
            int ok = 1;
            for (int a = 0; a < 3; ++a) {
                e[a] = r[a] + s6 * (((k1[a] + 2.0 * k2[a]) + 2.0 * k3[a]) + k4[a]);
                ok = ok && e[a] >= 0.0 && e[a] <= L[a];
            }
            if (!ok) break;
            for (int a = 0; a < 3; ++a) { r[a] = e[a]; out[3 * len + a] = e[a]; }
            ++len;
        }
        lengths[q] = len;
    }
}
