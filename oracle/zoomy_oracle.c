/*
 * zoomy_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the explicit finite-volume step of
 * the shallow-water / shallow-moment hierarchy (Eq. (sme), Sec. 1; the 2D SME
 * system and friction closure of Sec. 3.4; the hyperbolic predictor
 * Eq. (PDE-hyperbolic) and the source split Eq. (PDE-source), Sec. 2.1.2).
 *
 * It exists to check the GPU library.  Only the tests, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference leg may load it.  It shares no code,
 * header, table or constant with the CUDA path: the basis integrals are
 * computed here from the Legendre recurrence and Gauss-Legendre quadrature,
 * the mesh geometry and neighbours are rebuilt here from the raw mesh
 * description, and every model term is written out from its definition with
 * plain loops, cell by cell, each face evaluated from the side of the cell
 * being updated.  Compile with -ffp-contract=off.
 *
 * Readings of points where the paper is silent or inconsistent (all listed in
 * the design notes of the repository):
 *   R1 basis       phi_k(z) = P_k(1-2z): shifted Legendre, phi_k(0) = 1, z = 0 at the bed.
 *   R2 NC matrix   rows and columns k,l >= 1 only; row hA_k, column hA_l (x):
 *                  -u_m delta_kl + sum_{j>=1} alpha_j B_kjl / M_k with
 *                  B_kjl = <phi_k', phi_j Phi_l> (index order of Eq. (sme));
 *                  y-direction columns hB_l carry the same entries.
 *   R3 wave speed  s = |u_mean| + sqrt(g h + sum_{k>=1}|a_k|^2) + sum_{k>=2}|a_k|.
 *   R4 friction    slip  S_k = -(2k+1) (C/rho) u_b,  u_b = sum_k alpha_k (phi_k(0) = 1), k = 0..N;
 *                  Newtonian S_k = -(2k+1) (nu/(rho h)) sum_i C_ik alpha_i, C_ik = <phi_i', phi_k'>;
 *                  Manning bottom stress g n^2 |u_b| u_b / h^(1/3) in place of (C/rho) u_b.
 *   R5 time        SSP-RK2; per stage Y = X + dt L(X) with L = hyperbolic part + Newtonian
 *                  source at X; then the bottom stress as a linearly implicit cell-local
 *                  update (coefficient frozen at Y), then the dry cut.
 *   R6 scheme      path-conservative Rusanov with hydrostatic reconstruction: per face
 *                  |e| [ 1/2(F_n(Qi*)+F_n(Qj*)) - 1/2 s_f (Qj*-Qi*) - P(hi*) n
 *                        + 1/2 Btilde_n (Qj*-Qi*) ],  Btilde from 3-point Gauss-Legendre
 *                  along the straight segment in conserved variables.
 *   R7 CFL         dt = CFL * min_i Delta_i / max_i s_i,  Delta_i = 2|Omega_i|/P_i.
 *   R8 dry cells   velocities are zero where h <= h_dry (also along the NC path).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 8
#define OR_MAXM (OR_MAXN + 1)
#define OR_MAXV (1 + 2 * OR_MAXM)
#define OR_NQ 16 /* Gauss-Legendre points for the basis integrals (exact to degree 31) */

/* ------------------------------------------------------------------------- */
/* Legendre polynomials and the shifted basis (reading R1)                    */
/* ------------------------------------------------------------------------- */

/* P_0..P_n and their derivatives at x by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},   P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre_all(int n, double x, double *P, double *dP)
{
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n >= 1) {
        P[1] = x;
        dP[1] = 1.0;
    }
    for (int k = 1; k < n; ++k) {
        P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
        dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
    }
}

/* phi_k(z) = P_k(1-2z), phi_k'(z) = -2 P_k'(1-2z),
 * Phi_k(z) = int_0^z phi_k = z for k = 0, and for k >= 1, from
 * int P_k dx = (P_{k+1} - P_{k-1})/(2k+1) and dx = -2 dz:
 * Phi_k(z) = -(P_{k+1}(1-2z) - P_{k-1}(1-2z)) / (2(2k+1)). */
static void basis_eval(int N, double z, double *phi, double *dphi, double *Phi)
{
    double P[OR_MAXN + 3], dP[OR_MAXN + 3];
    double x = 1.0 - 2.0 * z;
    legendre_all(N + 1, x, P, dP);
    for (int k = 0; k <= N; ++k) {
        phi[k] = P[k];
        dphi[k] = -2.0 * dP[k];
        if (k == 0)
            Phi[k] = z;
        else
            Phi[k] = -(P[k + 1] - P[k - 1]) / (2.0 * (2.0 * k + 1.0));
    }
}

/* n-point Gauss-Legendre rule on [0,1] (Newton iteration on P_n). */
static void gauss_legendre01(int n, double *z, double *w)
{
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double P[64], dP[64];
        for (int it = 0; it < 100; ++it) {
            legendre_all(n, x, P, dP);
            double dx = P[n] / dP[n];
            x -= dx;
            if (fabs(dx) < 1e-15) { /* converged: one more Newton step polishes the last bits */
                legendre_all(n, x, P, dP);
                x -= P[n] / dP[n];
                break;
            }
        }
        legendre_all(n, x, P, dP);
        double wi = 2.0 / ((1.0 - x * x) * dP[n] * dP[n]);
        z[i] = 0.5 * (1.0 + x);
        w[i] = 0.5 * wi;
    }
}

/* Basis integrals (Sec. 2.1.1 "Basismatrices", Sec. 3.4):
 *   M[k]            = <phi_k, phi_k>
 *   A[(i*m+j)*m+k]  = <phi_i phi_j, phi_k>
 *   B[(k*m+j)*m+l]  = <phi_k', phi_j Phi_l>
 *   C[i*m+k]        = <phi_i', phi_k'>
 *   phi0[k]         = phi_k(0)
 * with m = N+1 and <f,g> = int_0^1 f g dz. */
int or_basis_tables(int N, double *M, double *A, double *B, double *C, double *phi0)
{
    if (N < 0 || N > OR_MAXN) return 1;
    int m = N + 1;
    double zq[OR_NQ], wq[OR_NQ];
    gauss_legendre01(OR_NQ, zq, wq);
    memset(M, 0, sizeof(double) * m);
    memset(A, 0, sizeof(double) * m * m * m);
    memset(B, 0, sizeof(double) * m * m * m);
    memset(C, 0, sizeof(double) * m * m);
    for (int q = 0; q < OR_NQ; ++q) {
        double phi[OR_MAXM], dphi[OR_MAXM], Phi[OR_MAXM];
        basis_eval(N, zq[q], phi, dphi, Phi);
        for (int i = 0; i < m; ++i) {
            M[i] += wq[q] * phi[i] * phi[i];
            for (int k = 0; k < m; ++k) C[i * m + k] += wq[q] * dphi[i] * dphi[k];
            for (int j = 0; j < m; ++j)
                for (int k = 0; k < m; ++k) {
                    A[(i * m + j) * m + k] += wq[q] * phi[i] * phi[j] * phi[k];
                    B[(i * m + j) * m + k] += wq[q] * dphi[i] * phi[j] * Phi[k];
                }
        }
    }
    /* Integrals that vanish by orthogonality or parity come out of the quadrature as
     * rounding noise of order 1e-17; every non-vanishing entry for N <= 8 exceeds 1e-6. */
    for (int i = 0; i < m * m * m; ++i) {
        if (fabs(A[i]) < 1e-13) A[i] = 0.0;
        if (fabs(B[i]) < 1e-13) B[i] = 0.0;
    }
    for (int i = 0; i < m * m; ++i)
        if (fabs(C[i]) < 1e-13) C[i] = 0.0;
    double phi[OR_MAXM], dphi[OR_MAXM], Phi[OR_MAXM];
    basis_eval(N, 0.0, phi, dphi, Phi);
    for (int k = 0; k < m; ++k) phi0[k] = phi[k];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Model (level N, dimension 1 or 2)                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int N, dim, nv, m;
    double g, h_dry;
    int fric; /* 0 none, 1 slip + Newtonian, 2 Manning */
    double C, nu, rho, manning_n;
    double M[OR_MAXM];
    double A[OR_MAXM * OR_MAXM * OR_MAXM];
    double B[OR_MAXM * OR_MAXM * OR_MAXM];
    double Cm[OR_MAXM * OR_MAXM];
    double phi0[OR_MAXM];
    int src_implicit; /* 0: reading R5 (explicit Newtonian, implicit bottom stress); 1: R17 */
    int order;        /* space order: 1 (reading R6) or 2 (reading R18, structured meshes) */
} or_model;

/* Variable order.  1D: (h, hA_0..hA_N).  2D: (h, hA_0, hB_0, hA_1..hA_N, hB_1..hB_N),
 * where hA_k = h alpha_k (x-velocity moments) and hB_k = h beta_k (y-velocity moments). */
static int ia(const or_model *md, int k)
{
    if (md->dim == 1) return 1 + k;
    return k == 0 ? 1 : 2 + k;
}
static int ib(const or_model *md, int k)
{
    return k == 0 ? 2 : 2 + md->N + k;
}

or_model *or_model_new(int N, int dim, double g, double h_dry, int fric, double C, double nu,
                       double rho, double manning_n)
{
    if (N < 0 || N > OR_MAXN || (dim != 1 && dim != 2)) return NULL;
    or_model *md = (or_model *)calloc(1, sizeof(or_model));
    md->N = N;
    md->dim = dim;
    md->m = N + 1;
    md->nv = dim == 1 ? 1 + md->m : 1 + 2 * md->m;
    md->g = g;
    md->h_dry = h_dry;
    md->fric = fric;
    md->C = C;
    md->nu = nu;
    md->rho = rho;
    md->manning_n = manning_n;
    md->order = 1;
    or_basis_tables(N, md->M, md->A, md->B, md->Cm, md->phi0);
    return md;
}
void or_model_free(or_model *md) { free(md); }
void or_model_set_source_mode(or_model *md, int mode) { md->src_implicit = mode; }
void or_model_set_order(or_model *md, int order) { md->order = order; }
int or_model_nv(const or_model *md) { return md->nv; }

/* Velocity moments alpha_k = hA_k / h, beta_k = hB_k / h; zero where h <= h_dry (R8). */
static void velocities(const or_model *md, const double *q, double *al, double *be)
{
    double h = q[0];
    for (int k = 0; k < md->m; ++k) {
        al[k] = 0.0;
        be[k] = 0.0;
        if (h > md->h_dry) {
            al[k] = q[ia(md, k)] / h;
            if (md->dim == 2) be[k] = q[ib(md, k)] / h;
        }
    }
}

/* Normal flux F_n = nx F_x + ny F_y (Eq. (sme) and the 2D SME flux of Sec. 3.4):
 *   h   row: h (alpha_0 nx + beta_0 ny)
 *   hA_k row: nx [h sum_ij alpha_i alpha_j A_ijk / M_k + delta_k0 g h^2/2] + ny h sum_ij beta_i alpha_j A_ijk / M_k
 *   hB_k row: nx h sum_ij alpha_i beta_j A_ijk / M_k + ny [h sum_ij beta_i beta_j A_ijk / M_k + delta_k0 g h^2/2] */
void or_flux(const or_model *md, const double *q, double nx, double ny, double *F)
{
    int m = md->m;
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    double h = q[0];
    for (int v = 0; v < md->nv; ++v) F[v] = 0.0;
    F[0] = h * al[0] * nx + (md->dim == 2 ? h * be[0] * ny : 0.0);
    for (int k = 0; k < m; ++k) {
        double saa = 0.0, sab = 0.0, sba = 0.0, sbb = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double a = md->A[(i * m + j) * m + k];
                saa += al[i] * al[j] * a;
                sab += al[i] * be[j] * a;
                sba += be[i] * al[j] * a;
                sbb += be[i] * be[j] * a;
            }
        double p = (k == 0) ? 0.5 * md->g * h * h : 0.0;
        F[ia(md, k)] = nx * (h * saa / md->M[k] + p);
        if (md->dim == 2) {
            F[ia(md, k)] += ny * (h * sba / md->M[k]);
            F[ib(md, k)] = nx * (h * sab / md->M[k]) + ny * (h * sbb / md->M[k] + p);
        }
    }
}

/* Nonconservative matrix B_n = nx B_x + ny B_y, row-major nv x nv (reading R2). */
void or_nc_matrix(const or_model *md, const double *q, double nx, double ny, double *Bn)
{
    int m = md->m, nv = md->nv;
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    for (int v = 0; v < nv * nv; ++v) Bn[v] = 0.0;
    for (int k = 1; k < m; ++k)
        for (int l = 1; l < m; ++l) {
            double ea = (k == l) ? -al[0] : 0.0; /* -u_m delta_kl */
            double eb = (k == l) ? -be[0] : 0.0; /* -v_m delta_kl */
            for (int j = 1; j < m; ++j) {
                ea += al[j] * md->B[(k * m + j) * m + l] / md->M[k];
                eb += be[j] * md->B[(k * m + j) * m + l] / md->M[k];
            }
            /* x-direction: columns hA_l */
            Bn[ia(md, k) * nv + ia(md, l)] += nx * ea;
            if (md->dim == 2) {
                Bn[ib(md, k) * nv + ia(md, l)] += nx * eb;
                /* y-direction: columns hB_l */
                Bn[ia(md, k) * nv + ib(md, l)] += ny * ea;
                Bn[ib(md, k) * nv + ib(md, l)] += ny * eb;
            }
        }
}

/* Cell wave-speed bound (reading R3). */
double or_wavespeed(const or_model *md, const double *q)
{
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    double h = q[0] > 0.0 ? q[0] : 0.0;
    double um = sqrt(al[0] * al[0] + be[0] * be[0]);
    double s2 = 0.0, s1 = 0.0;
    for (int k = 1; k < md->m; ++k) {
        double ak2 = al[k] * al[k] + be[k] * be[k];
        s2 += ak2;
        if (k >= 2) s1 += sqrt(ak2);
    }
    return um + sqrt(md->g * h + s2) + s1;
}

/* Newtonian bulk friction (reading R4), explicit part of the source. */
void or_source_newtonian(const or_model *md, const double *q, double *S)
{
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    for (int v = 0; v < md->nv; ++v) S[v] = 0.0;
    if (md->fric != 1 || !(q[0] > md->h_dry)) return;
    double h = q[0];
    for (int k = 0; k < md->m; ++k) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < md->m; ++i) {
            sa += al[i] * md->Cm[i * md->m + k];
            sb += be[i] * md->Cm[i * md->m + k];
        }
        S[ia(md, k)] = -(md->nu / (md->rho * h)) * sa / md->M[k];
        if (md->dim == 2) S[ib(md, k)] = -(md->nu / (md->rho * h)) * sb / md->M[k];
    }
}

/* Bottom stress, linearly implicit (reading R5), then the dry cut (R8), in place.
 * The stress on row k is -(phi_k(0)/M_k) c sum_i hA_i with c = C/(rho h) (slip) or
 * c = g n^2 |u_b| / h^(4/3) (Manning), frozen at the input state y.  The implicit
 * system z + dt c w (1^T z) = y, w_k = phi_k(0)/M_k, is solved by the Sherman-Morrison
 * formula z = y - dt c w (1^T y) / (1 + dt c 1^T w). */
void or_bottom_friction(const or_model *md, double *y, double dt)
{
    double h = y[0];
    int m = md->m;
    if (!(h > md->h_dry)) {
        for (int v = 1; v < md->nv; ++v) y[v] = 0.0;
        return;
    }
    if (md->fric == 0) return;
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < m; ++k) {
        sa += md->phi0[k] * y[ia(md, k)];
        if (md->dim == 2) sb += md->phi0[k] * y[ib(md, k)];
    }
    double c;
    if (md->fric == 1) {
        c = md->C / (md->rho * h);
    } else {
        double ub = sa / h, vb = sb / h;
        double n2 = md->manning_n * md->manning_n;
        c = md->g * n2 * sqrt(ub * ub + vb * vb) / pow(h, 4.0 / 3.0);
    }
    double sw = 0.0;
    for (int k = 0; k < m; ++k) sw += md->phi0[k] / md->M[k];
    double den = 1.0 + dt * c * sw;
    for (int k = 0; k < m; ++k) {
        double w = md->phi0[k] / md->M[k];
        y[ia(md, k)] -= dt * c * w * sa / den;
        if (md->dim == 2) y[ib(md, k)] -= dt * c * w * sb / den;
    }
}

/* ------------------------------------------------------------------------- */
/* Mesh (built here from the raw description, independent of the library)    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t nc;
    int nf;          /* faces per cell: 2 (1D), 4 (quads), 3 (triangles) */
    int dim;
    double *area;    /* |Omega_i| */
    double *delta;   /* 2 |Omega_i| / P_i */
    int64_t *nbr;    /* [nc*nf], -1 on the boundary */
    double *fnx, *fny, *flen; /* outward unit normal and length per (cell, face) */
    int *fbc;        /* boundary kind per (cell, face): 0 transmissive, 1 wall */
} or_mesh;

static or_mesh *mesh_alloc(int64_t nc, int nf, int dim)
{
    or_mesh *me = (or_mesh *)calloc(1, sizeof(or_mesh));
    me->nc = nc;
    me->nf = nf;
    me->dim = dim;
    me->area = (double *)calloc(nc, sizeof(double));
    me->delta = (double *)calloc(nc, sizeof(double));
    me->nbr = (int64_t *)calloc(nc * nf, sizeof(int64_t));
    me->fnx = (double *)calloc(nc * nf, sizeof(double));
    me->fny = (double *)calloc(nc * nf, sizeof(double));
    me->flen = (double *)calloc(nc * nf, sizeof(double));
    me->fbc = (int *)calloc(nc * nf, sizeof(int));
    return me;
}

void or_mesh_free(or_mesh *me)
{
    if (!me) return;
    free(me->area);
    free(me->delta);
    free(me->nbr);
    free(me->fnx);
    free(me->fny);
    free(me->flen);
    free(me->fbc);
    free(me);
}

int64_t or_mesh_ncells(const or_mesh *me) { return me->nc; }

/* Uniform 1D grid on [x0,x1]; bc_left, bc_right in {0 transmissive, 1 wall}. */
or_mesh *or_mesh_1d(int64_t nx, double x0, double x1, int bc_left, int bc_right)
{
    or_mesh *me = mesh_alloc(nx, 2, 1);
    double dx = (x1 - x0) / (double)nx;
    for (int64_t i = 0; i < nx; ++i) {
        me->area[i] = dx;
        me->delta[i] = 2.0 * dx / 2.0;
        me->nbr[i * 2 + 0] = i - 1;
        me->fnx[i * 2 + 0] = -1.0;
        me->flen[i * 2 + 0] = 1.0;
        me->fbc[i * 2 + 0] = bc_left;
        me->nbr[i * 2 + 1] = (i + 1 < nx) ? i + 1 : -1;
        me->fnx[i * 2 + 1] = 1.0;
        me->flen[i * 2 + 1] = 1.0;
        me->fbc[i * 2 + 1] = bc_right;
    }
    return me;
}

/* nx x ny rectangles on [x0,x1] x [y0,y1], cell (i,j) at index j*nx + i.
 * bc = {x-, x+, y-, y+}. */
or_mesh *or_mesh_2d(int64_t nx, int64_t ny, double x0, double x1, double y0, double y1,
                    const int *bc)
{
    or_mesh *me = mesh_alloc(nx * ny, 4, 2);
    double dx = (x1 - x0) / (double)nx, dy = (y1 - y0) / (double)ny;
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t c = j * nx + i, f = c * 4;
            me->area[c] = dx * dy;
            me->delta[c] = 2.0 * dx * dy / (2.0 * dx + 2.0 * dy);
            me->nbr[f + 0] = i > 0 ? c - 1 : -1;
            me->fnx[f + 0] = -1.0; me->fny[f + 0] = 0.0; me->flen[f + 0] = dy; me->fbc[f + 0] = bc[0];
            me->nbr[f + 1] = i + 1 < nx ? c + 1 : -1;
            me->fnx[f + 1] = 1.0; me->fny[f + 1] = 0.0; me->flen[f + 1] = dy; me->fbc[f + 1] = bc[1];
            me->nbr[f + 2] = j > 0 ? c - nx : -1;
            me->fnx[f + 2] = 0.0; me->fny[f + 2] = -1.0; me->flen[f + 2] = dx; me->fbc[f + 2] = bc[2];
            me->nbr[f + 3] = j + 1 < ny ? c + nx : -1;
            me->fnx[f + 3] = 0.0; me->fny[f + 3] = 1.0; me->flen[f + 3] = dx; me->fbc[f + 3] = bc[3];
        }
    return me;
}

typedef struct {
    int64_t a, b; /* sorted vertex pair */
    int64_t cell;
    int face;
} half_edge;

static int cmp_half_edge(const void *x, const void *y)
{
    const half_edge *p = (const half_edge *)x, *q = (const half_edge *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/* Triangles (vertex indices into verts_xy[2*nverts]); every boundary edge gets kind bc. */
or_mesh *or_mesh_tri(int64_t nverts, const double *xy, int64_t ntris, const int32_t *tris, int bc)
{
    or_mesh *me = mesh_alloc(ntris, 3, 2);
    half_edge *he = (half_edge *)malloc(sizeof(half_edge) * 3 * ntris);
    for (int64_t t = 0; t < ntris; ++t) {
        int64_t v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        double sa = 0.5 * ((xy[2 * v[1]] - xy[2 * v[0]]) * (xy[2 * v[2] + 1] - xy[2 * v[0] + 1]) -
                           (xy[2 * v[2]] - xy[2 * v[0]]) * (xy[2 * v[1] + 1] - xy[2 * v[0] + 1]));
        if (sa < 0.0) { /* make the triangle counter-clockwise */
            int64_t tmp = v[1];
            v[1] = v[2];
            v[2] = tmp;
            sa = -sa;
        }
        double per = 0.0;
        for (int f = 0; f < 3; ++f) {
            int64_t p = v[f], q = v[(f + 1) % 3];
            double ex = xy[2 * q] - xy[2 * p], ey = xy[2 * q + 1] - xy[2 * p + 1];
            double len = sqrt(ex * ex + ey * ey);
            me->fnx[t * 3 + f] = ey / len; /* outward normal of a CCW edge p->q */
            me->fny[t * 3 + f] = -ex / len;
            me->flen[t * 3 + f] = len;
            me->fbc[t * 3 + f] = bc;
            me->nbr[t * 3 + f] = -1;
            per += len;
            he[3 * t + f].a = p < q ? p : q;
            he[3 * t + f].b = p < q ? q : p;
            he[3 * t + f].cell = t;
            he[3 * t + f].face = f;
        }
        me->area[t] = sa;
        me->delta[t] = 2.0 * sa / per;
    }
    qsort(he, 3 * ntris, sizeof(half_edge), cmp_half_edge);
    for (int64_t e = 0; e + 1 < 3 * ntris; ++e) {
        if (he[e].a == he[e + 1].a && he[e].b == he[e + 1].b) {
            me->nbr[he[e].cell * 3 + he[e].face] = he[e + 1].cell;
            me->nbr[he[e + 1].cell * 3 + he[e + 1].face] = he[e].cell;
            ++e;
        }
    }
    free(he);
    (void)nverts;
    return me;
}

/* Geometry accessors (for the tests). */
void or_mesh_geometry(const or_mesh *me, double *area, double *delta, int64_t *nbr, double *fnx,
                      double *fny, double *flen)
{
    memcpy(area, me->area, sizeof(double) * me->nc);
    memcpy(delta, me->delta, sizeof(double) * me->nc);
    memcpy(nbr, me->nbr, sizeof(int64_t) * me->nc * me->nf);
    memcpy(fnx, me->fnx, sizeof(double) * me->nc * me->nf);
    memcpy(fny, me->fny, sizeof(double) * me->nc * me->nf);
    memcpy(flen, me->flen, sizeof(double) * me->nc * me->nf);
}

/* ------------------------------------------------------------------------- */
/* The finite-volume step                                                      */
/* ------------------------------------------------------------------------- */

static void gather(const double *Q, int64_t nc, int nv, int64_t i, double *q)
{
    for (int v = 0; v < nv; ++v) q[v] = Q[(int64_t)v * nc + i];
}

/* Ghost state across a boundary face: transmissive copies the cell; a wall keeps h
 * and reflects every velocity-moment vector, a_k -> a_k - 2 (a_k . n) n. */
static void ghost(const or_model *md, const double *qi, int bc, double nx, double ny, double *qg)
{
    for (int v = 0; v < md->nv; ++v) qg[v] = qi[v];
    if (bc != 1) return;
    for (int k = 0; k < md->m; ++k) {
        if (md->dim == 1) {
            qg[ia(md, k)] = -qi[ia(md, k)];
        } else {
            double a = qi[ia(md, k)], b = qi[ib(md, k)];
            double an = a * nx + b * ny;
            qg[ia(md, k)] = a - 2.0 * an * nx;
            qg[ib(md, k)] = b - 2.0 * an * ny;
        }
    }
}

/* Hydrostatic reconstruction of a cell state against the face bed level bf:
 * h* = max(0, h + b - bf), velocities kept (zero if h <= h_dry or h* <= h_dry). */
static void hydrostatic_state(const or_model *md, const double *q, double b, double bf, double *qs)
{
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    double hs = q[0] + b - bf;
    if (hs < 0.0) hs = 0.0;
    for (int v = 0; v < md->nv; ++v) qs[v] = 0.0;
    qs[0] = hs;
    if (!(hs > md->h_dry)) return;
    for (int k = 0; k < md->m; ++k) {
        qs[ia(md, k)] = hs * al[k];
        if (md->dim == 2) qs[ib(md, k)] = hs * be[k];
    }
}

/* The face term of reading R6, seen from cell i (outward normal n, length len is
 * applied by the caller):  1/2(F_n(Qi*)+F_n(Qj*)) - 1/2 s_f (Qj*-Qi*) - P(hi*) n
 *                         + 1/2 Btilde_n (Qj*-Qi*). */
static void face_term(const or_model *md, const double *qi, double bi, const double *qj,
                      double bj, double nx, double ny, double *out)
{
    int nv = md->nv;
    double bf = bi > bj ? bi : bj;
    double qsi[OR_MAXV], qsj[OR_MAXV], Fi[OR_MAXV], Fj[OR_MAXV], dq[OR_MAXV];
    hydrostatic_state(md, qi, bi, bf, qsi);
    hydrostatic_state(md, qj, bj, bf, qsj);
    or_flux(md, qsi, nx, ny, Fi);
    or_flux(md, qsj, nx, ny, Fj);
    double si = or_wavespeed(md, qsi), sj = or_wavespeed(md, qsj);
    double sf = si > sj ? si : sj;
    for (int v = 0; v < nv; ++v) {
        dq[v] = qsj[v] - qsi[v];
        out[v] = 0.5 * (Fi[v] + Fj[v]) - 0.5 * sf * dq[v];
    }
    double p = 0.5 * md->g * qsi[0] * qsi[0];
    out[ia(md, 0)] -= p * nx;
    if (md->dim == 2) out[ib(md, 0)] -= p * ny;

    /* 3-point Gauss-Legendre on [0,1] along Psi(s) = Qi* + s (Qj* - Qi*) */
    const double sq[3] = {0.5 - sqrt(15.0) / 10.0, 0.5, 0.5 + sqrt(15.0) / 10.0};
    const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    double Bt[OR_MAXV * OR_MAXV], Bq[OR_MAXV * OR_MAXV], psi[OR_MAXV];
    for (int v = 0; v < nv * nv; ++v) Bt[v] = 0.0;
    for (int q = 0; q < 3; ++q) {
        for (int v = 0; v < nv; ++v) psi[v] = qsi[v] + sq[q] * dq[v];
        or_nc_matrix(md, psi, nx, ny, Bq);
        for (int v = 0; v < nv * nv; ++v) Bt[v] += wq[q] * Bq[v];
    }
    for (int r = 0; r < nv; ++r) {
        double acc = 0.0;
        for (int c = 0; c < nv; ++c) acc += Bt[r * nv + c] * dq[c];
        out[r] += 0.5 * acc;
    }
}

/* One explicit stage Y = R(X + dt L(X)) (readings R5, R6). */
/* Friction fully implicit (reading R17, the paper's step_source_implicit for Eq. (PDE-source)):
 * backward Euler on dy/dt = -K y for the moment rows y_k = h alpha_k (and h beta_k), with
 *   K_ki = (phi_k(0)/M_k) c phi_i(0) + (nu / (rho h^2)) C_ik / M_k,
 * the bottom stress (c = C/(rho h), or Manning's g n^2 |u_b| / h^(4/3)) and the Newtonian bulk
 * stress (slip + Newtonian only), h and c frozen at the input y.  (I + dt K) z = y is solved by
 * Gaussian elimination with partial pivoting; then the dry cut (R8), in place. */
void or_friction_implicit(const or_model *md, double *y, double dt)
{
    double h = y[0];
    int m = md->m;
    if (!(h > md->h_dry)) {
        for (int v = 1; v < md->nv; ++v) y[v] = 0.0;
        return;
    }
    if (md->fric == 0) return;
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < m; ++k) {
        sa += md->phi0[k] * y[ia(md, k)];
        if (md->dim == 2) sb += md->phi0[k] * y[ib(md, k)];
    }
    double c;
    if (md->fric == 1) {
        c = md->C / (md->rho * h);
    } else {
        double ub = sa / h, vb = sb / h;
        c = md->g * md->manning_n * md->manning_n * sqrt(ub * ub + vb * vb) / pow(h, 4.0 / 3.0);
    }
    double nuh = md->fric == 1 ? md->nu / (md->rho * h * h) : 0.0;
    double A[OR_MAXM][OR_MAXM + 2]; /* augmented: two right-hand sides (alpha rows, beta rows) */
    for (int k = 0; k < m; ++k) {
        for (int i = 0; i < m; ++i)
            A[k][i] = (k == i ? 1.0 : 0.0) +
                      dt * (md->phi0[k] / md->M[k] * c * md->phi0[i] + nuh * md->Cm[i * m + k] / md->M[k]);
        A[k][m] = y[ia(md, k)];
        A[k][m + 1] = md->dim == 2 ? y[ib(md, k)] : 0.0;
    }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < m + 2; ++j) {
                double t = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = t;
            }
        for (int r = col + 1; r < m; ++r) {
            double f = A[r][col] / A[col][col];
            for (int j = col; j < m + 2; ++j) A[r][j] -= f * A[col][j];
        }
    }
    for (int rhs = 0; rhs < 2; ++rhs) {
        double z[OR_MAXM];
        for (int k = m - 1; k >= 0; --k) {
            double s = A[k][m + rhs];
            for (int j = k + 1; j < m; ++j) s -= A[k][j] * z[j];
            z[k] = s / A[k][k];
        }
        for (int k = 0; k < m; ++k) {
            if (rhs == 0) y[ia(md, k)] = z[k];
            else if (md->dim == 2) y[ib(md, k)] = z[k];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Second order in space (reading R18): MUSCL on 1D and structured 2D meshes   */
/* ------------------------------------------------------------------------- */

static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* Reconstruction variables of a state: w = (h, eta = h + b, alpha_0..alpha_N, beta_0..beta_N). */
static int prim_vars(const or_model *md, const double *q, double b, double *w)
{
    double al[OR_MAXM], be[OR_MAXM];
    velocities(md, q, al, be);
    w[0] = q[0];
    w[1] = q[0] + b;
    for (int k = 0; k < md->m; ++k) {
        w[2 + k] = al[k];
        if (md->dim == 2) w[2 + md->m + k] = be[k];
    }
    return md->dim == 2 ? 2 + 2 * md->m : 2 + md->m;
}

/* Neighbour of cell i across its face f (state and bed), the ghost of A9 on boundary faces. */
static void neighbour(const or_model *md, const or_mesh *me, const double *X, const double *bed, int64_t i,
                      int f, double *qj, double *bj)
{
    double qi[OR_MAXV];
    int64_t e = i * me->nf + f, j = me->nbr[e];
    if (j >= 0) {
        gather(X, me->nc, md->nv, j, qj);
        *bj = bed ? bed[j] : 0.0;
    } else {
        gather(X, me->nc, md->nv, i, qi);
        ghost(md, qi, me->fbc[e], me->fnx[e], me->fny[e], qj);
        *bj = bed ? bed[i] : 0.0;
    }
}

/* Limited slopes of cell i in direction d (faces 2d and 2d+1 of the cell): sigma = minmod of the
 * one-sided differences of w, zero for every variable if one of the three cells is dry. */
static void slopes(const or_model *md, const or_mesh *me, const double *X, const double *bed, int64_t i, int d,
                   double *sig)
{
    double qi[OR_MAXV], ql[OR_MAXV], qr[OR_MAXV], wi[2 + 2 * OR_MAXM], wl[2 + 2 * OR_MAXM], wr[2 + 2 * OR_MAXM];
    double bl, br;
    gather(X, me->nc, md->nv, i, qi);
    neighbour(md, me, X, bed, i, 2 * d, ql, &bl);
    neighbour(md, me, X, bed, i, 2 * d + 1, qr, &br);
    int nw = prim_vars(md, qi, bed ? bed[i] : 0.0, wi);
    prim_vars(md, ql, bl, wl);
    prim_vars(md, qr, br, wr);
    int dry = !(qi[0] > md->h_dry) || !(ql[0] > md->h_dry) || !(qr[0] > md->h_dry);
    for (int v = 0; v < nw; ++v) sig[v] = dry ? 0.0 : minmod(wi[v] - wl[v], wr[v] - wi[v]);
}

/* Face state of cell i on side s (-1: face 2d, +1: face 2d+1) of direction d:
 * w + s sigma / 2, the bed b + s (sigma_eta - sigma_h) / 2, as a conserved state. */
static void face_state(const or_model *md, const double *qi, double bi, const double *sig, int s, double *qf,
                       double *bf)
{
    double w[2 + 2 * OR_MAXM];
    int nw = prim_vars(md, qi, bi, w);
    for (int v = 0; v < nw; ++v) w[v] += 0.5 * s * sig[v];
    *bf = bi + 0.5 * s * (sig[1] - sig[0]);
    for (int v = 0; v < md->nv; ++v) qf[v] = 0.0;
    qf[0] = w[0];
    for (int k = 0; k < md->m; ++k) {
        qf[ia(md, k)] = w[0] * w[2 + k];
        if (md->dim == 2) qf[ib(md, k)] = w[0] * w[2 + md->m + k];
    }
}

/* Second-order hyperbolic part of cell i: sum over faces of |e| times the face term between the
 * two reconstructed face states, plus per direction the cell-interior terms
 *   |e_d| g (h_+ + h_-)/2 (eta_+ - eta_-)                on the normal mean-momentum row,
 *   |e_d| Btilde_d(Q_- -> Q_+) (Q_+ - Q_-)               (3-point Gauss-Legendre path integral),
 * which vanish for zero slopes (first order) and for a lake at rest. */
static void hyperbolic2(const or_model *md, const or_mesh *me, const double *X, const double *bed, int64_t i,
                        double *acc)
{
    int nv = md->nv, ndir = me->nf / 2;
    double qi[OR_MAXV], term[OR_MAXV];
    gather(X, me->nc, nv, i, qi);
    double bi = bed ? bed[i] : 0.0;
    for (int v = 0; v < nv; ++v) acc[v] = 0.0;
    for (int d = 0; d < ndir; ++d) {
        double sig[2 + 2 * OR_MAXM], qm[OR_MAXV], qp[OR_MAXV], bm, bp;
        slopes(md, me, X, bed, i, d, sig);
        face_state(md, qi, bi, sig, -1, qm, &bm);
        face_state(md, qi, bi, sig, +1, qp, &bp);
        for (int side = 0; side < 2; ++side) {
            int f = 2 * d + side;
            int64_t e = i * me->nf + f, j = me->nbr[e];
            const double *qf = side ? qp : qm;
            double bf = side ? bp : bm, qn[OR_MAXV], bn;
            if (j >= 0) {
                double qjc[OR_MAXV], sj[2 + 2 * OR_MAXM];
                gather(X, me->nc, nv, j, qjc);
                slopes(md, me, X, bed, j, d, sj);
                face_state(md, qjc, bed ? bed[j] : 0.0, sj, side ? -1 : +1, qn, &bn);
            } else {
                ghost(md, qf, me->fbc[e], me->fnx[e], me->fny[e], qn);
                bn = bf;
            }
            face_term(md, qf, bf, qn, bn, me->fnx[e], me->fny[e], term);
            for (int v = 0; v < nv; ++v) acc[v] += me->flen[e] * term[v];
        }
        /* cell interior, normal +e_d, face length of direction d */
        double len = me->flen[i * me->nf + 2 * d], nx = d == 0 ? 1.0 : 0.0, ny = d == 0 ? 0.0 : 1.0;
        double etap = qp[0] + bp, etam = qm[0] + bm;
        int row = d == 0 ? ia(md, 0) : ib(md, 0);
        acc[row] += len * 0.5 * md->g * (qp[0] + qm[0]) * (etap - etam);
        const double sq[3] = {0.5 - sqrt(15.0) / 10.0, 0.5, 0.5 + sqrt(15.0) / 10.0};
        const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
        double Bt[OR_MAXV * OR_MAXV], Bq[OR_MAXV * OR_MAXV], psi[OR_MAXV], dq[OR_MAXV];
        for (int v = 0; v < nv; ++v) dq[v] = qp[v] - qm[v];
        for (int v = 0; v < nv * nv; ++v) Bt[v] = 0.0;
        for (int q = 0; q < 3; ++q) {
            for (int v = 0; v < nv; ++v) psi[v] = qm[v] + sq[q] * dq[v];
            or_nc_matrix(md, psi, nx, ny, Bq);
            for (int v = 0; v < nv * nv; ++v) Bt[v] += wq[q] * Bq[v];
        }
        for (int r = 0; r < nv; ++r) {
            double a = 0.0;
            for (int c = 0; c < nv; ++c) a += Bt[r * nv + c] * dq[c];
            acc[r] += len * a;
        }
    }
}

void or_stage(const or_model *md, const or_mesh *me, const double *X, const double *bed, double dt,
              double *Y)
{
    int nv = md->nv;
    int64_t nc = me->nc;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nc; ++i) {
        double qi[OR_MAXV], qj[OR_MAXV], term[OR_MAXV], acc[OR_MAXV], S[OR_MAXV], y[OR_MAXV];
        gather(X, nc, nv, i, qi);
        double bi = bed ? bed[i] : 0.0;
        for (int v = 0; v < nv; ++v) acc[v] = 0.0;
        if (md->order == 2 && me->nf != 3) {
            hyperbolic2(md, me, X, bed, i, acc);
        } else {
            for (int f = 0; f < me->nf; ++f) {
                int64_t e = i * me->nf + f;
                double nx = me->fnx[e], ny = me->fny[e], bj;
                int64_t j = me->nbr[e];
                if (j >= 0) {
                    gather(X, nc, nv, j, qj);
                    bj = bed ? bed[j] : 0.0;
                } else {
                    ghost(md, qi, me->fbc[e], nx, ny, qj);
                    bj = bi;
                }
                face_term(md, qi, bi, qj, bj, nx, ny, term);
                for (int v = 0; v < nv; ++v) acc[v] += me->flen[e] * term[v];
            }
        }
        if (md->src_implicit) {
            for (int v = 0; v < nv; ++v) y[v] = qi[v] - dt / me->area[i] * acc[v];
            or_friction_implicit(md, y, dt);
        } else {
            or_source_newtonian(md, qi, S);
            for (int v = 0; v < nv; ++v) y[v] = qi[v] - dt / me->area[i] * acc[v] + dt * S[v];
            or_bottom_friction(md, y, dt);
        }
        for (int v = 0; v < nv; ++v) Y[(int64_t)v * nc + i] = y[v];
    }
}

double or_max_wavespeed(const or_model *md, const or_mesh *me, const double *Q)
{
    double smax = 0.0;
    double q[OR_MAXV];
    for (int64_t i = 0; i < me->nc; ++i) {
        gather(Q, me->nc, md->nv, i, q);
        double s = or_wavespeed(md, q);
        if (s > smax || s != s) smax = s;
    }
    return smax;
}

double or_min_delta(const or_mesh *me)
{
    double d = me->delta[0];
    for (int64_t i = 1; i < me->nc; ++i)
        if (me->delta[i] < d) d = me->delta[i];
    return d;
}

/* Time step of reading R7 for the state Q. */
double or_cfl_dt(const or_model *md, const or_mesh *me, const double *Q, double cfl)
{
    return cfl * or_min_delta(me) / or_max_wavespeed(md, me, Q);
}

/* Precision form of the FP32 state: the state is kept in single precision between stages while
 * every operation on it is FP64.  store_f32 != 0 rounds Q1 and Q^{n+1} to the nearest float at
 * the points where an FP32-state implementation stores them. */
static void round_to_float(double *a, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) a[k] = (double)(float)a[k];
}

/* nsteps SSP-RK2 steps: Q1 = stage(Qn), Q2 = stage(Q1), Qn+1 = (Qn + Q2)/2.
 * dt_fixed > 0 uses that step; dt_fixed <= 0 recomputes dt from Qn every step.
 * Q is [nv][nc]; bed may be NULL (flat).  Returns the time advanced in *t_out. */
int or_step_ex(const or_model *md, const or_mesh *me, double *Q, const double *bed, double dt_fixed,
               double cfl, int nsteps, int store_f32, double *t_out)
{
    int64_t n = (int64_t)md->nv * me->nc;
    double *Q1 = (double *)malloc(sizeof(double) * n);
    double *Q2 = (double *)malloc(sizeof(double) * n);
    double t = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = dt_fixed > 0.0 ? dt_fixed : or_cfl_dt(md, me, Q, cfl);
        or_stage(md, me, Q, bed, dt, Q1);
        if (store_f32) round_to_float(Q1, n);
        or_stage(md, me, Q1, bed, dt, Q2);
        for (int64_t k = 0; k < n; ++k) Q[k] = 0.5 * (Q[k] + Q2[k]);
        if (store_f32) round_to_float(Q, n);
        t += dt;
    }
    free(Q1);
    free(Q2);
    if (t_out) *t_out = t;
    return 0;
}

int or_step(const or_model *md, const or_mesh *me, double *Q, const double *bed, double dt_fixed,
            double cfl, int nsteps, double *t_out)
{
    return or_step_ex(md, me, Q, bed, dt_fixed, cfl, nsteps, 0, t_out);
}

/* Total mass sum_i |Omega_i| h_i (FP64). */
double or_mass(const or_mesh *me, const double *Q)
{
    double s = 0.0;
    for (int64_t i = 0; i < me->nc; ++i) s += me->area[i] * Q[i];
    return s;
}

int or_max_level(void) { return OR_MAXN; }

/* ------------------------------------------------------------------------- */
/* Lifting to three-dimensional fields (Sec. "Postprocessing": interpolate_3d) */
/* ------------------------------------------------------------------------- */

/* Reading R16.  At sigma levels zeta_j in [0,1] (elevation z = b + zeta h):
 *   u(zeta) = sum_k alpha_k phi_k(zeta),  v(zeta) = sum_k beta_k phi_k(zeta)   (the moment expansion);
 *   w(zeta) from continuity, integrated upwards from the bed where w = u.grad b:
 *     w = -d_x(int_b^z u dz') - d_y(int_b^z v dz')  at fixed z, with int_b^z u dz' = sum_k hA_k Phi_k(zeta),
 *     so w(zeta) = -sum_k [d_x hA_k + d_y hB_k] Phi_k(zeta) + u(zeta)(d_x b + zeta d_x h)
 *                  + v(zeta)(d_y b + zeta d_y h);
 *   p(zeta) = g h (1 - zeta)   (hydrostatic, rho = 1).
 * Level 0 on a flat bed at zeta = 1 gives the paper's SWE lifting w = -h (d_x u + d_y v).
 * Horizontal derivatives: Green-Gauss over the cell's faces, face value (q_i + q_j)/2 with q_j = q_i on
 * boundary faces.  Dry cells (h <= h_dry): u = v = w = 0.  bed may be NULL (flat).
 * out: [4][K][nc] = u, v, w, p. */
void or_lift3d(const or_model *md, const or_mesh *me, const double *Q, const double *bed, int K,
               const double *zeta, double *out)
{
    const int64_t nc = me->nc;
    const int m = md->m, nv = md->nv;
    for (int64_t i = 0; i < nc; ++i) {
        double gx[OR_MAXV + 1], gy[OR_MAXV + 1]; /* d/dx, d/dy of every variable and (index nv) of b */
        for (int v = 0; v <= nv; ++v) gx[v] = gy[v] = 0.0;
        for (int f = 0; f < me->nf; ++f) {
            const int64_t j = me->nbr[i * me->nf + f];
            const double wx = me->flen[i * me->nf + f] * me->fnx[i * me->nf + f];
            const double wy = me->flen[i * me->nf + f] * me->fny[i * me->nf + f];
            for (int v = 0; v <= nv; ++v) {
                const double qi = v < nv ? Q[v * nc + i] : (bed ? bed[i] : 0.0);
                const double qj = j < 0 ? qi : (v < nv ? Q[v * nc + j] : (bed ? bed[j] : 0.0));
                const double fv = 0.5 * (qi + qj);
                gx[v] += wx * fv;
                gy[v] += wy * fv;
            }
        }
        for (int v = 0; v <= nv; ++v) {
            gx[v] /= me->area[i];
            gy[v] /= me->area[i];
        }
        double q[OR_MAXV], al[OR_MAXM], be[OR_MAXM];
        for (int v = 0; v < nv; ++v) q[v] = Q[v * nc + i];
        velocities(md, q, al, be);
        const double h = q[0];
        const int wet = h > md->h_dry;
        for (int jz = 0; jz < K; ++jz) {
            double phi[OR_MAXM], dphi[OR_MAXM], Phi[OR_MAXM];
            basis_eval(md->N, zeta[jz], phi, dphi, Phi);
            double u = 0.0, v = 0.0, G = 0.0;
            for (int k = 0; k < m; ++k) {
                u += al[k] * phi[k];
                v += be[k] * phi[k];
                G += gx[ia(md, k)] * Phi[k];
                if (md->dim == 2) G += gy[ib(md, k)] * Phi[k];
            }
            double w = -G + u * (gx[nv] + zeta[jz] * gx[0]) + v * (gy[nv] + zeta[jz] * gy[0]);
            if (!wet) u = v = w = 0.0;
            out[(0 * K + jz) * nc + i] = u;
            out[(1 * K + jz) * nc + i] = v;
            out[(2 * K + jz) * nc + i] = w;
            out[(3 * K + jz) * nc + i] = md->g * h * (1.0 - zeta[jz]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Learned closure (level-1 prognostic state, level-4 model)                  */
/* ------------------------------------------------------------------------- */
/*
 * Reading: the closure model is the level-4 system restricted to the rows of the level-1
 * variables (h, hA_0, hB_0, hA_1, hB_1); the velocity moments alpha_k, beta_k of k = 2..4 come
 * from a per-cell MLP of the level-1 state at every stage input (features h, u_m, v_m, alpha_1,
 * beta_1, lambda scaled by in_scale; outputs scaled by out_scale).  Face terms are the level-4 ones
 * on the closed states, projected on the level-1 rows; the Newtonian source sums over all five
 * moments; the bottom stress is implicit in the two prognostic moments with the closed moments
 * frozen at the stage input; the CFL speed is the level-4 bound on the closed state.
 * Schedule (reading R21): the network is evaluated on every stage input (schedule 0), or once per
 * step on Q^n with its predicted velocity moments held for both stages (schedule 1): a stage input X
 * then closes with alpha_hat(Q^n), cut to zero where X is dry, and its own depth.
 * GELU: tanh form.  bf16 != 0 rounds each layer input to BF16 (nearest, ties to even) like the
 * tensor-core inference kernel; all arithmetic is FP64.
 */
typedef struct {
    double W1[6 * 64], b1[64], W2[64 * 64], b2[64], W3[64 * 6], b3[6];
    double in_scale[6], out_scale[6];
    int bf16;
} or_closure;

or_closure *or_closure_new(const double *params, const double *in_scale, const double *out_scale, int bf16)
{
    or_closure *c = (or_closure *)calloc(1, sizeof(or_closure));
    const double *p = params;
    memcpy(c->W1, p, sizeof(c->W1)); p += 6 * 64;
    memcpy(c->b1, p, sizeof(c->b1)); p += 64;
    memcpy(c->W2, p, sizeof(c->W2)); p += 64 * 64;
    memcpy(c->b2, p, sizeof(c->b2)); p += 64;
    memcpy(c->W3, p, sizeof(c->W3)); p += 64 * 6;
    memcpy(c->b3, p, sizeof(c->b3));
    memcpy(c->in_scale, in_scale, sizeof(c->in_scale));
    memcpy(c->out_scale, out_scale, sizeof(c->out_scale));
    c->bf16 = bf16;
    return c;
}
void or_closure_free(or_closure *c) { free(c); }

static double round_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double gelu_tanh(double z)
{
    const double c = 0.79788456080286535588; /* sqrt(2/pi) */
    return 0.5 * z * (1.0 + tanh(c * (z + 0.044715 * z * z * z)));
}

/* features (h, u_m, v_m, alpha_1, beta_1, lambda) -> (alpha_2, alpha_3, alpha_4, beta_2, beta_3, beta_4) */
void or_closure_eval(const or_closure *c, const double *feat, double *out)
{
    double x[6], a1[64], a2[64];
    for (int i = 0; i < 6; ++i) {
        x[i] = feat[i] * c->in_scale[i];
        if (c->bf16) x[i] = round_bf16(x[i]);
    }
    for (int j = 0; j < 64; ++j) {
        double z = c->b1[j];
        for (int i = 0; i < 6; ++i) z += x[i] * c->W1[i * 64 + j];
        a1[j] = gelu_tanh(z);
        if (c->bf16) a1[j] = round_bf16(a1[j]);
    }
    for (int j = 0; j < 64; ++j) {
        double z = c->b2[j];
        for (int i = 0; i < 64; ++i) z += a1[i] * c->W2[i * 64 + j];
        a2[j] = gelu_tanh(z);
        if (c->bf16) a2[j] = round_bf16(a2[j]);
    }
    for (int j = 0; j < 6; ++j) {
        double z = c->b3[j];
        for (int i = 0; i < 64; ++i) z += a2[i] * c->W3[i * 6 + j];
        out[j] = z * c->out_scale[j];
    }
}

/* The predicted velocity moments (alpha_2..4, beta_2..4) of a level-1 state q1 (variables h, hA0,
 * hB0, hA1, hB1); lambda is the slip feature. */
static void closure_predict(const or_model *m4, const or_closure *c, const double *q1, double lambda, double *out)
{
    double h = q1[0];
    double u = 0.0, v = 0.0, a1 = 0.0, b1 = 0.0;
    if (h > m4->h_dry) {
        u = q1[1] / h;
        v = q1[2] / h;
        a1 = q1[3] / h;
        b1 = q1[4] / h;
    }
    double feat[6] = {h, u, v, a1, b1, lambda};
    or_closure_eval(c, feat, out);
}

/* The closed level-4 state of q1 with predicted velocity moments pred (zero where q1 is dry).
 * Returns the closed moments in alpha_hat / beta_hat (k = 2..4). */
static void closure_close(const or_model *m4, const double *q1, const double *pred, double *q4, double *ahat,
                          double *bhat)
{
    double h = q1[0];
    for (int v2 = 0; v2 < m4->nv; ++v2) q4[v2] = 0.0;
    q4[0] = h;
    q4[ia(m4, 0)] = q1[1];
    q4[ib(m4, 0)] = q1[2];
    q4[ia(m4, 1)] = q1[3];
    q4[ib(m4, 1)] = q1[4];
    for (int k = 2; k <= 4; ++k) {
        ahat[k] = h > m4->h_dry ? pred[k - 2] : 0.0;
        bhat[k] = h > m4->h_dry ? pred[k + 1] : 0.0;
        q4[ia(m4, k)] = h * ahat[k];
        q4[ib(m4, k)] = h * bhat[k];
    }
}

static void closure_embed(const or_model *m4, const or_closure *c, const double *q1, double lambda, double *q4,
                          double *ahat, double *bhat)
{
    double out[6];
    closure_predict(m4, c, q1, lambda, out);
    closure_close(m4, q1, out, q4, ahat, bhat);
}

/* One closure stage Y = R(X + dt L(X)) on the level-1 state X [5][nc]. */
/* pred: the predicted moments [nc][6] to close X with (schedule 1), or NULL to predict from X. */
static void closure_stage(const or_model *m4, const or_closure *cl, const or_mesh *me, const double *X,
                          const double *bed, double dt, const double *pred, double *Y)
{
    int64_t nc = me->nc;
    double *X4 = (double *)malloc(sizeof(double) * (size_t)m4->nv * nc);
    double *sig = (double *)malloc(sizeof(double) * 2 * nc); /* sum_{k>=2} alpha_hat, beta_hat */
    for (int64_t i = 0; i < nc; ++i) {
        double q1[5], q4[OR_MAXV], ah[5], bh[5];
        for (int v = 0; v < 5; ++v) q1[v] = X[(int64_t)v * nc + i];
        if (pred)
            closure_close(m4, q1, pred + 6 * i, q4, ah, bh);
        else
            closure_embed(m4, cl, q1, m4->C, q4, ah, bh);
        for (int v = 0; v < m4->nv; ++v) X4[(int64_t)v * nc + i] = q4[v];
        sig[2 * i] = ah[2] + ah[3] + ah[4];
        sig[2 * i + 1] = bh[2] + bh[3] + bh[4];
    }
    const int rows[5] = {0, ia(m4, 0), ib(m4, 0), ia(m4, 1), ib(m4, 1)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nc; ++i) {
        double qi[OR_MAXV], qj[OR_MAXV], term[OR_MAXV], acc[OR_MAXV], S[OR_MAXV];
        gather(X4, nc, m4->nv, i, qi);
        double bi = bed ? bed[i] : 0.0;
        for (int v = 0; v < m4->nv; ++v) acc[v] = 0.0;
        for (int f = 0; f < me->nf; ++f) {
            int64_t e = i * me->nf + f;
            double nx = me->fnx[e], ny = me->fny[e], bj;
            int64_t j = me->nbr[e];
            if (j >= 0) {
                gather(X4, nc, m4->nv, j, qj);
                bj = bed ? bed[j] : 0.0;
            } else {
                ghost(m4, qi, me->fbc[e], nx, ny, qj);
                bj = bi;
            }
            face_term(m4, qi, bi, qj, bj, nx, ny, term);
            for (int v = 0; v < m4->nv; ++v) acc[v] += me->flen[e] * term[v];
        }
        or_source_newtonian(m4, qi, S);
        double y[5];
        for (int r = 0; r < 5; ++r) y[r] = X[(int64_t)r * nc + i] - dt / me->area[i] * acc[rows[r]] + dt * S[rows[r]];
        /* bottom stress: implicit in the prognostic moments (rows 1..4), closed moments frozen */
        double h = y[0];
        if (!(h > m4->h_dry)) {
            y[1] = y[2] = y[3] = y[4] = 0.0;
        } else if (m4->fric != 0) {
            double sa_hat = h * sig[2 * i], sb_hat = h * sig[2 * i + 1];
            double c;
            if (m4->fric == 1) {
                c = m4->C / (m4->rho * h);
            } else {
                double ub = (y[1] + y[3] + sa_hat) / h, vb = (y[2] + y[4] + sb_hat) / h;
                c = m4->g * m4->manning_n * m4->manning_n * sqrt(ub * ub + vb * vb) / pow(h, 4.0 / 3.0);
            }
            /* rows (hA0, hA1) with weights w = (1, 3): z + dt c w (z0 + z1) = y - dt c w sa_hat */
            double ra0 = y[1] - dt * c * 1.0 * sa_hat, ra1 = y[3] - dt * c * 3.0 * sa_hat;
            double rb0 = y[2] - dt * c * 1.0 * sb_hat, rb1 = y[4] - dt * c * 3.0 * sb_hat;
            double den = 1.0 + dt * c * 4.0;
            double fa = dt * c * (ra0 + ra1) / den, fb = dt * c * (rb0 + rb1) / den;
            y[1] = ra0 - 1.0 * fa;
            y[3] = ra1 - 3.0 * fa;
            y[2] = rb0 - 1.0 * fb;
            y[4] = rb1 - 3.0 * fb;
        }
        for (int r = 0; r < 5; ++r) Y[(int64_t)r * nc + i] = y[r];
    }
    free(X4);
    free(sig);
}

/* Max level-4 wave speed of the closed state of Q1. */
double or_closure_max_wavespeed(const or_model *m4, const or_closure *cl, const or_mesh *me, const double *Q1)
{
    double smax = 0.0;
    for (int64_t i = 0; i < me->nc; ++i) {
        double q1[5], q4[OR_MAXV], ah[5], bh[5];
        for (int v = 0; v < 5; ++v) q1[v] = Q1[(int64_t)v * me->nc + i];
        closure_embed(m4, cl, q1, m4->C, q4, ah, bh);
        double s = or_wavespeed(m4, q4);
        if (s > smax || s != s) smax = s;
    }
    return smax;
}

/* nsteps SSP-RK2 steps of the closure model on the level-1 state Q1 [5][nc]; m4 is the level-4 2D
 * model (its C is the slip coefficient and the lambda feature).  store_f32 as in or_step_ex;
 * schedule as in the header of this section. */
int or_step_closure(const or_model *m4, const or_closure *cl, const or_mesh *me, double *Q1, const double *bed,
                    double dt_fixed, double cfl, int nsteps, int store_f32, int schedule, double *t_out)
{
    if (m4->N != 4 || m4->dim != 2 || schedule < 0 || schedule > 1) return 1;
    int64_t n = 5 * me->nc;
    double *A = (double *)malloc(sizeof(double) * n);
    double *B = (double *)malloc(sizeof(double) * n);
    double *P = schedule == 1 ? (double *)malloc(sizeof(double) * 6 * me->nc) : NULL;
    double t = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = dt_fixed > 0.0 ? dt_fixed : cfl * or_min_delta(me) / or_closure_max_wavespeed(m4, cl, me, Q1);
        if (P) {
            for (int64_t i = 0; i < me->nc; ++i) {
                double q1[5];
                for (int v = 0; v < 5; ++v) q1[v] = Q1[(int64_t)v * me->nc + i];
                closure_predict(m4, cl, q1, m4->C, P + 6 * i);
            }
        }
        closure_stage(m4, cl, me, Q1, bed, dt, P, A);
        if (store_f32) round_to_float(A, n);
        closure_stage(m4, cl, me, A, bed, dt, P, B);
        for (int64_t k = 0; k < n; ++k) Q1[k] = 0.5 * (Q1[k] + B[k]);
        if (store_f32) round_to_float(Q1, n);
        t += dt;
    }
    free(A);
    free(B);
    free(P);
    if (t_out) *t_out = t;
    return 0;
}
