/*
 * oracle.c -- plain, slow CPU reference (FP64) for the block-hydro packet task.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: it is compiled separately (oracle/build.py) and used by tests/,
 * the smoke check and the CPU-baseline leg of the benchmark. It shares no
 * source with the CUDA library (no headers, helpers or constants).
 *
 * What it computes. The paper's GPU task function (section "Code Generators":
 * a group of API calls run on one device with no transfer in between) runs on
 * a data packet of n concatenated mesh blocks (section "DataItem Generators").
 * Every block has the same cell count and a uniform cell size (section
 * "Flash-X"); a halo of guard cells is refreshed before the task (section
 * "Experiments", Spark paragraph); the gas is ideal gamma-law (section "Sedov
 * Blast Wave", EOS sentence). The paper prints no formulas for the solver
 * beyond "explicit finite volume"; the scheme written out below is:
 *   guard fill -> primitives -> minmod slopes -> Hancock half-step predictor
 *   -> face states -> HLL (Davis wave speeds) fluxes -> unsplit conservative
 *   update, with dt = CFL / max_cells sum_d (|u_d| + c) / dx_d.
 * A second integrator, for the paper's Spark solver ("explicit finite
 * volume, 2nd-order Runge-Kutta", section "Experiments"): Heun's two-stage
 * method with the same steps minus the half-step predictor (ora_step_rk2).
 * Each step is a function below, in that order, with plain loops over blocks
 * and cells; unstated details are fixed by the "Reading:" notes in place.
 *
 * Arithmetic contract: every floating-point expression is written with its
 * evaluation order made explicit by parentheses; the file must be compiled
 * without FMA contraction (-ffp-contract=off) so the results are the IEEE
 * FP64 value of exactly these expressions.
 *
 * Data layout of a state array U (input and output): interior cells only,
 * [block][var][k][j][i], i fastest; block id = bx + nbx*(by + nby*bz);
 * vars = (rho, m_x, m_y[, m_z], E). 2D meshes use nb[2] = bs[2] = 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 2        /* guard cells per side (two-cell stencil of MUSCL-Hancock) */
#define MAXV 5     /* max conserved vars (3D) */

typedef struct {
    int ndim;          /* 2 or 3 */
    int nb[3];         /* blocks per axis (nb[2] = 1 in 2D) */
    int bs[3];         /* interior cells per block per axis (bs[2] = 1 in 2D) */
    int periodic[3];   /* per axis: 1 periodic, 0 outflow (zero-gradient) */
    double gamma;      /* ratio of specific heats */
    double cfl;        /* Courant number of the summed-direction CFL rule */
    double lo[3], hi[3];
} ora_mesh;

static int nvars(const ora_mesh* m) { return m->ndim + 2; }
static long ncell_block(const ora_mesh* m) { return (long)m->bs[0] * m->bs[1] * m->bs[2]; }
static long nblocks(const ora_mesh* m) { return (long)m->nb[0] * m->nb[1] * m->nb[2]; }

static double cell_width(const ora_mesh* m, int d) {
    return (m->hi[d] - m->lo[d]) / (double)(m->nb[d] * m->bs[d]);
}

/* ---------------------------------------------------------------- guard fill
 * Value of conserved variable v at global cell (gi, gj, gk), where indices may
 * lie outside the domain. Reading of "outflow": zero-gradient, i.e. the index
 * is clamped to [0, N-1] on each axis independently (faces, edges and corners
 * alike); periodic axes wrap instead. */
static int map_index(int gi, int n, int periodic) {
    if (periodic) { gi %= n; if (gi < 0) gi += n; return gi; }
    if (gi < 0) return 0;
    if (gi > n - 1) return n - 1;
    return gi;
}

static double global_value(const ora_mesh* m, const double* U, int v, int gi, int gj, int gk) {
    int g[3] = {gi, gj, gk};
    int bidx[3], loc[3];
    for (int d = 0; d < 3; ++d) {
        int n = m->nb[d] * m->bs[d];
        int c = (d < m->ndim) ? map_index(g[d], n, m->periodic[d]) : 0;
        bidx[d] = c / m->bs[d];
        loc[d] = c % m->bs[d];
    }
    long b = bidx[0] + (long)m->nb[0] * (bidx[1] + (long)m->nb[1] * bidx[2]);
    long off = ((long)loc[2] * m->bs[1] + loc[1]) * m->bs[0] + loc[0];
    return U[(b * nvars(m) + v) * ncell_block(m) + off];
}

/* ---------------------------------------------------------------- EOS / primitives
 * W = (rho, u_x, u_y[, u_z], p) from U = (rho, m_x, m_y[, m_z], E):
 *   r = 1/rho, u_d = m_d * r, p = (gamma - 1) * (E - 0.5 * sum_d m_d u_d).
 * Also returns r (used again by the predictor). */
static void prim_from_cons(int ndim, double gamma, const double* U, double* W, double* r_out) {
    int nv = ndim + 2;
    double rho = U[0];
    double r = 1.0 / rho;
    double mu = 0.0;
    W[0] = rho;
    for (int d = 0; d < ndim; ++d) {
        W[1 + d] = U[1 + d] * r;
        mu = (d == 0) ? (U[1] * W[1]) : (mu + (U[1 + d] * W[1 + d]));
    }
    double ke = 0.5 * mu;
    W[nv - 1] = (gamma - 1.0) * (U[nv - 1] - ke);
    *r_out = r;
}

/* U from W: m_d = rho * u_d, E = p / (gamma - 1) + (0.5 rho) |u|^2, with
 * 1/(gamma-1) formed once. */
static void cons_from_prim(int ndim, double gamma, const double* W, double* U) {
    int nv = ndim + 2;
    double rho = W[0], p = W[nv - 1];
    double q2 = 0.0;
    U[0] = rho;
    for (int d = 0; d < ndim; ++d) {
        U[1 + d] = rho * W[1 + d];
        q2 = (d == 0) ? (W[1] * W[1]) : (q2 + (W[1 + d] * W[1 + d]));
    }
    double igm1 = 1.0 / (gamma - 1.0);
    U[nv - 1] = (p * igm1) + ((0.5 * rho) * q2);
}

/* ---------------------------------------------------------------- limiter
 * minmod(a, b): the smaller-magnitude argument when both have the same strict
 * sign, else 0. Written with sign tests (no a*b product). */
double ora_minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return (a < b) ? a : b;
    if (a < 0.0 && b < 0.0) return (a > b) ? a : b;
    return 0.0;
}

/* ---------------------------------------------------------------- HLL flux
 * Flux across a face with normal axis d between left state WL and right state
 * WR (primitives). Davis wave-speed estimates
 *   S_L = min(u_L - c_L, u_R - c_R),  S_R = max(u_L + c_L, u_R + c_R),
 * with c = sqrt(gamma p / rho) written as sqrt((gamma*p) * (1/rho)).
 *   S_L >= 0: F = F(U_L);  S_R <= 0: F = F(U_R);
 *   else F = ((S_R F_L - S_L F_R) + (S_L S_R)(U_R - U_L)) * (1 / (S_R - S_L)).
 * Physical flux along d: (m_d, m_k u_d [+ p if k == d], (E + p) u_d). */
static void phys_flux(int ndim, int d, const double* W, const double* U, double* F) {
    int nv = ndim + 2;
    double un = W[1 + d], p = W[nv - 1];
    F[0] = U[1 + d];
    for (int k = 0; k < ndim; ++k) {
        F[1 + k] = (k == d) ? ((U[1 + k] * un) + p) : (U[1 + k] * un);
    }
    F[nv - 1] = (U[nv - 1] + p) * un;
}

void ora_hll(int ndim, int d, double gamma, const double* WL, const double* WR, double* F) {
    int nv = ndim + 2;
    double UL[MAXV], UR[MAXV], FL[MAXV], FR[MAXV];
    double cL = sqrt((gamma * WL[nv - 1]) * (1.0 / WL[0]));
    double cR = sqrt((gamma * WR[nv - 1]) * (1.0 / WR[0]));
    double a = WL[1 + d] - cL, b = WR[1 + d] - cR;
    double SL = (a < b) ? a : b;
    a = WL[1 + d] + cL; b = WR[1 + d] + cR;
    double SR = (a > b) ? a : b;
    cons_from_prim(ndim, gamma, WL, UL);
    cons_from_prim(ndim, gamma, WR, UR);
    phys_flux(ndim, d, WL, UL, FL);
    phys_flux(ndim, d, WR, UR, FR);
    if (SL >= 0.0) { memcpy(F, FL, sizeof(double) * nv); return; }
    if (SR <= 0.0) { memcpy(F, FR, sizeof(double) * nv); return; }
    double slsr = SL * SR;
    double inv = 1.0 / (SR - SL);
    for (int v = 0; v < nv; ++v) {
        F[v] = (((SR * FL[v]) - (SL * FR[v])) + (slsr * (UR[v] - UL[v]))) * inv;
    }
}

/* ---------------------------------------------------------------- CFL time step
 * Signal speed of one cell: s = sum_d (|u_d| + c) * (1/dx_d), summed x, y, z.
 * Reading of "CFL 0.8": the sum over directions (stable for the unsplit
 * update without transverse corrections), not the per-direction minimum. */
static double cell_signal_speed(const ora_mesh* m, const double* Ucell, const double* idx) {
    double W[MAXV], r;
    int nv = nvars(m);
    prim_from_cons(m->ndim, m->gamma, Ucell, W, &r);
    double c = sqrt((m->gamma * W[nv - 1]) * r);
    double s = 0.0;
    for (int d = 0; d < m->ndim; ++d) {
        double sd = (fabs(W[1 + d]) + c) * idx[d];
        s = (d == 0) ? sd : (s + sd);
    }
    return s;
}

/* Largest signal speed over all interior cells; returns -1 if any cell has a
 * non-positive or non-finite density or pressure. */
double ora_max_signal_speed(const ora_mesh* m, const double* U) {
    int nv = nvars(m);
    long nc = ncell_block(m), nblk = nblocks(m);
    double idx[3];
    for (int d = 0; d < 3; ++d) idx[d] = 1.0 / cell_width(m, d);
    double smax = 0.0;
    int bad = 0;
    for (long b = 0; b < nblk; ++b) {
        for (long c = 0; c < nc; ++c) {
            double Uc[MAXV], W[MAXV], r;
            for (int v = 0; v < nv; ++v) Uc[v] = U[(b * nv + v) * nc + c];
            prim_from_cons(m->ndim, m->gamma, Uc, W, &r);
            if (!(W[0] > 0.0) || !(W[nv - 1] > 0.0)) bad = 1;
            double s = cell_signal_speed(m, Uc, idx);
            if (s > smax) smax = s;
        }
    }
    return bad ? -1.0 : smax;
}

double ora_dt(const ora_mesh* m, const double* U) {
    double s = ora_max_signal_speed(m, U);
    if (!(s > 0.0)) return -1.0;
    return m->cfl / s;
}

/* ---------------------------------------------------------------- one block
 * Padded work arrays of one block: index (i, j, k) with i in [-G, bs0+G),
 * likewise j and k (k only in 3D). */
typedef struct {
    int p[3];          /* padded extents */
    int off[3];        /* offset of local index 0 (G, or 0 on an unused axis) */
    double* U;         /* [v][pk][pj][pi] conserved incl. guards */
    double* W;         /* [v][...] primitives */
    double* R;         /* [...] 1/rho */
    double* FS;        /* [cell][d][side][v] face states (side 0: low face, 1: high face) */
    int* first;        /* [cell] 1 if the cell fell back to first order */
    const struct ora_amr_src* amr;  /* fine level of a two-level mesh: where cells come from (else NULL) */
    double* reg;       /* NULL, or this block's face fluxes [2d + side][v][face cell] (flux register) */
    long out_b;        /* block index of the output (-1: the block's own index) */
} ora_work;

static double amr_value(const struct ora_amr_src* s, int v, int gi, int gj, int gk);

static long pidx(const ora_work* w, int i, int j, int k) {
    return ((long)(k + w->off[2]) * w->p[1] + (j + w->off[1])) * w->p[0] + (i + w->off[0]);
}

/* Flux registers: index of the face cell of (i, j, k) on a face normal to
 * axis d (the two other axes, lower one fastest), and the stride between
 * faces (the largest face of a block). */
static long face_cell(const ora_mesh* m, int d, const int loc[3]) {
    int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
    return (long)loc[a2] * m->bs[a1] + loc[a1];
}

static long face_stride(const ora_mesh* m) {
    long f = 0;
    for (int d = 0; d < 3; ++d) {
        int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
        long n = (long)m->bs[a1] * m->bs[a2];
        if (n > f) f = n;
    }
    return f;
}

/* Fill the padded conserved array of block (bx, by, bz) from the global state:
 * interior cells and guard cells alike read global_value(), which applies the
 * boundary rule on the domain edge and reads the neighbour block otherwise. */
static void fill_padded_block(const ora_mesh* m, const double* U, int bxyz[3], ora_work* w) {
    int nv = nvars(m);
    long np = (long)w->p[0] * w->p[1] * w->p[2];
    for (int k = -w->off[2]; k < w->p[2] - w->off[2]; ++k)
        for (int j = -w->off[1]; j < w->p[1] - w->off[1]; ++j)
            for (int i = -w->off[0]; i < w->p[0] - w->off[0]; ++i) {
                int gi = bxyz[0] * m->bs[0] + i;
                int gj = bxyz[1] * m->bs[1] + j;
                int gk = bxyz[2] * m->bs[2] + k;
                for (int v = 0; v < nv; ++v)
                    w->U[v * np + pidx(w, i, j, k)] =
                        w->amr ? amr_value(w->amr, v, gi, gj, gk) : global_value(m, U, v, gi, gj, gk);
            }
}

/* Advance one block by dt: reads the global state U (for guards), writes the
 * block's interior into Unew, accumulates domain-boundary fluxes into bflux
 * (units of the cell sum: sum_faces c_d * F, + on the high side, - on the low
 * side), counts first-order cells and non-physical primitives.
 * predictor = 1: MUSCL-Hancock (face states from the half-step state);
 * predictor = 0: plain MUSCL (face states from the stage's own primitives),
 * the spatial operator of the Runge-Kutta stages. Ubase = NULL: Unew = U - acc
 * (a forward-Euler stage, or the Hancock step); else the second Heun stage
 * Unew = 0.5 * (Ubase + (U - acc)), Ubase read at the cell only. */
static void advance_block(const ora_mesh* m, const double* U, const double* Ubase, int predictor, double dt,
                          long b, double* Unew, double* bflux, long* nfirst, long* nbad, ora_work* w) {
    int nv = nvars(m), nd = m->ndim;
    double g = m->gamma;
    int bxyz[3] = {(int)(b % m->nb[0]), (int)((b / m->nb[0]) % m->nb[1]), (int)(b / ((long)m->nb[0] * m->nb[1]))};
    long np = (long)w->p[0] * w->p[1] * w->p[2];
    double idx[3], cd[3], hd[3];
    for (int d = 0; d < 3; ++d) {
        idx[d] = 1.0 / cell_width(m, d);
        cd[d] = dt * idx[d];     /* dt / dx_d */
        hd[d] = 0.5 * cd[d];     /* (dt/2) / dx_d */
    }
    int lo[3], hi[3];            /* cell range where face states are formed: [-1, bs] on active axes */
    for (int d = 0; d < 3; ++d) {
        lo[d] = (d < nd) ? -1 : 0;
        hi[d] = (d < nd) ? m->bs[d] : 0;
    }
    int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

    /* 1. guard fill */
    fill_padded_block(m, U, bxyz, w);

    /* 2. primitives on the whole padded block */
    for (long c = 0; c < np; ++c) {
        double Uc[MAXV], Wc[MAXV], r;
        for (int v = 0; v < nv; ++v) Uc[v] = w->U[v * np + c];
        prim_from_cons(nd, g, Uc, Wc, &r);
        for (int v = 0; v < nv; ++v) w->W[v * np + c] = Wc[v];
        w->R[c] = r;
    }
    /* interior cells must be physical */
    for (int k = 0; k < m->bs[2]; ++k)
        for (int j = 0; j < m->bs[1]; ++j)
            for (int i = 0; i < m->bs[0]; ++i) {
                long c = pidx(w, i, j, k);
                if (!(w->W[c] > 0.0) || !(w->W[(nv - 1) * np + c] > 0.0)) (*nbad)++;
            }

    /* 3-5. slopes, Hancock predictor and face states on [-1, bs] per axis */
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                long c = pidx(w, i, j, k);
                double Wc[MAXV], dW[3][MAXV], a[3][MAXV], Wbar[MAXV];
                for (int v = 0; v < nv; ++v) Wc[v] = w->W[v * np + c];
                double rc = w->R[c];
                /* 3. minmod slopes of the primitives, per axis and component */
                for (int d = 0; d < nd; ++d) {
                    long cm = pidx(w, i - e[d][0], j - e[d][1], k - e[d][2]);
                    long cp = pidx(w, i + e[d][0], j + e[d][1], k + e[d][2]);
                    for (int v = 0; v < nv; ++v) {
                        double dl = Wc[v] - w->W[v * np + cm];
                        double dr = w->W[v * np + cp] - Wc[v];
                        dW[d][v] = ora_minmod(dl, dr);
                    }
                }
                /* 4. Hancock predictor in primitive form, summed over all axes:
                 *    Wbar = W - sum_d (dt/2)/dx_d * A_d(W) dW_d, where along axis d
                 *    with normal velocity u_n:
                 *      rho: u_n drho + rho du_n
                 *      u_n: u_n du_n + dp * (1/rho)
                 *      u_t: u_n du_t
                 *      p:   (gamma p) du_n + u_n dp                              */
                double gp = g * Wc[nv - 1];
                for (int d = 0; d < nd && predictor; ++d) {
                    double un = Wc[1 + d];
                    double dun = dW[d][1 + d], dp = dW[d][nv - 1];
                    a[d][0] = (un * dW[d][0]) + (Wc[0] * dun);
                    for (int t = 0; t < nd; ++t)
                        a[d][1 + t] = (t == d) ? ((un * dun) + (dp * rc)) : (un * dW[d][1 + t]);
                    a[d][nv - 1] = (gp * dun) + (un * dp);
                }
                for (int v = 0; v < nv; ++v) {
                    if (!predictor) { Wbar[v] = Wc[v]; continue; }     /* plain MUSCL: no half step */
                    double s = 0.0;
                    for (int d = 0; d < nd; ++d)
                        s = (d == 0) ? (hd[0] * a[0][v]) : (s + (hd[d] * a[d][v]));
                    Wbar[v] = Wc[v] - s;
                }
                /* 5. face states Wbar -+ dW/2. Reading: if any face state of the
                 *    cell has rho <= 0 or p <= 0, the whole cell reverts to first
                 *    order (all its face states equal W). */
                double* fs = w->FS + c * (3 * 2 * MAXV);
                int ok = 1;
                for (int d = 0; d < nd; ++d)
                    for (int v = 0; v < nv; ++v) {
                        double hs = 0.5 * dW[d][v];
                        fs[(d * 2 + 0) * MAXV + v] = Wbar[v] - hs;
                        fs[(d * 2 + 1) * MAXV + v] = Wbar[v] + hs;
                    }
                for (int d = 0; d < nd; ++d)
                    for (int s = 0; s < 2; ++s) {
                        const double* q = fs + (d * 2 + s) * MAXV;
                        if (!(q[0] > 0.0) || !(q[nv - 1] > 0.0)) ok = 0;
                    }
                if (!ok) {
                    for (int d = 0; d < nd; ++d)
                        for (int s = 0; s < 2; ++s)
                            for (int v = 0; v < nv; ++v) fs[(d * 2 + s) * MAXV + v] = Wc[v];
                }
                w->first[c] = !ok;
            }
    for (int k = 0; k < m->bs[2]; ++k)
        for (int j = 0; j < m->bs[1]; ++j)
            for (int i = 0; i < m->bs[0]; ++i) *nfirst += w->first[pidx(w, i, j, k)];

    /* 6-7. HLL fluxes on both faces of every interior cell, and the unsplit
     *      update U+ = U - [c_x (Fx_hi - Fx_lo) + c_y (..) + c_z (..)], summed
     *      x, y, z. A face's flux depends only on the two face states, so the
     *      same face evaluated from either side gives the same value. */
    for (int k = 0; k < m->bs[2]; ++k)
        for (int j = 0; j < m->bs[1]; ++j)
            for (int i = 0; i < m->bs[0]; ++i) {
                long c = pidx(w, i, j, k);
                double acc[MAXV];
                for (int d = 0; d < nd; ++d) {
                    long cm = pidx(w, i - e[d][0], j - e[d][1], k - e[d][2]);
                    long cp = pidx(w, i + e[d][0], j + e[d][1], k + e[d][2]);
                    const double* fsc = w->FS + c * (3 * 2 * MAXV);
                    const double* fsm = w->FS + cm * (3 * 2 * MAXV);
                    const double* fsp = w->FS + cp * (3 * 2 * MAXV);
                    double Flo[MAXV], Fhi[MAXV];
                    ora_hll(nd, d, g, fsm + (d * 2 + 1) * MAXV, fsc + (d * 2 + 0) * MAXV, Flo);
                    ora_hll(nd, d, g, fsc + (d * 2 + 1) * MAXV, fsp + (d * 2 + 0) * MAXV, Fhi);
                    for (int v = 0; v < nv; ++v) {
                        double t = cd[d] * (Fhi[v] - Flo[v]);
                        acc[v] = (d == 0) ? t : (acc[v] + t);
                    }
                    /* domain-boundary flux bookkeeping (outflow axes only) */
                    int loc[3] = {i, j, k};
                    if (w->reg) {    /* flux register: the fluxes through the block's own faces */
                        long t = face_cell(m, d, loc);
                        long fsz = face_stride(m);
                        if (loc[d] == 0)
                            for (int v = 0; v < nv; ++v) w->reg[((2 * d) * MAXV + v) * fsz + t] = Flo[v];
                        if (loc[d] == m->bs[d] - 1)
                            for (int v = 0; v < nv; ++v) w->reg[((2 * d + 1) * MAXV + v) * fsz + t] = Fhi[v];
                    }
                    if (!m->periodic[d]) {
                        if (bxyz[d] == 0 && loc[d] == 0)
                            for (int v = 0; v < nv; ++v) bflux[v] -= cd[d] * Flo[v];
                        if (bxyz[d] == m->nb[d] - 1 && loc[d] == m->bs[d] - 1)
                            for (int v = 0; v < nv; ++v) bflux[v] += cd[d] * Fhi[v];
                    }
                }
                long co = ((long)k * m->bs[1] + j) * m->bs[0] + i;
                for (int v = 0; v < nv; ++v) {
                    long o = ((w->out_b >= 0 ? w->out_b : b) * nv + v) * ncell_block(m) + co;
                    double us = w->U[v * np + c] - acc[v];
                    Unew[o] = Ubase ? (0.5 * (Ubase[o] + us)) : us;
                }
            }
}

static int n_threads = 1;

void ora_set_threads(int n) { n_threads = (n < 1) ? 1 : n; }

int ora_get_threads(void) { return n_threads; }

/* One pass of advance_block over every block (see there for predictor and
 * Ubase). bflux (nvar doubles, may be NULL) receives the boundary-flux total;
 * returns the number of first-order cells, or -1 if an interior cell had
 * rho <= 0 or p <= 0. */
static long sweep(const ora_mesh* m, const double* U, const double* Ubase, int predictor, double dt, double* Unew,
                  double* bflux) {
    int nv = nvars(m);
    long nblk = nblocks(m);
    long nfirst = 0, nbad = 0;
    double* bf_all = (double*)calloc((size_t)nblk * MAXV, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads) reduction(+ : nfirst, nbad)
#endif
    {
        ora_work w;
        for (int d = 0; d < 3; ++d) {
            w.off[d] = (d < m->ndim) ? G : 0;
            w.p[d] = m->bs[d] + 2 * w.off[d];
        }
        long np = (long)w.p[0] * w.p[1] * w.p[2];
        w.U = (double*)malloc(sizeof(double) * np * MAXV);
        w.W = (double*)malloc(sizeof(double) * np * MAXV);
        w.R = (double*)malloc(sizeof(double) * np);
        w.FS = (double*)malloc(sizeof(double) * np * 3 * 2 * MAXV);
        w.first = (int*)calloc((size_t)np, sizeof(int));
        w.amr = NULL;
        w.reg = NULL;
        w.out_b = -1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long b = 0; b < nblk; ++b)
            advance_block(m, U, Ubase, predictor, dt, b, Unew, bf_all + b * MAXV, &nfirst, &nbad, &w);
        free(w.U); free(w.W); free(w.R); free(w.FS); free(w.first);
    }
    if (bflux) {
        for (int v = 0; v < nv; ++v) {
            double s = 0.0;
            for (long b = 0; b < nblk; ++b) s += bf_all[b * MAXV + v];
            bflux[v] = s;
        }
    }
    free(bf_all);
    return nbad ? -1 : nfirst;
}

/* One MUSCL-Hancock time step of every block: Unew = step(U, dt); bflux and
 * the return value as for sweep(). */
long ora_step(const ora_mesh* m, const double* U, double dt, double* Unew, double* bflux) {
    return sweep(m, U, NULL, 1, dt, Unew, bflux);
}

/* One Runge-Kutta stage with the plain MUSCL operator L (no half step):
 * Ubase = NULL: Unew = U + dt L(U) (the first Heun stage); else
 * Unew = 0.5 * (Ubase + (U + dt L(U))) (the second). */
long ora_stage(const ora_mesh* m, const double* U, const double* Ubase, double dt, double* Unew, double* bflux) {
    return sweep(m, U, Ubase, 0, dt, Unew, bflux);
}

/* One step of Heun's two-stage Runge-Kutta method (the strong-stability-
 * preserving RK2 of Shu and Osher) with the plain MUSCL operator:
 *   U* = U + dt L(U),   Unew = 0.5 * (U + (U* + dt L(U*))),
 * guards refreshed from each stage's own state. bflux receives
 * 0.5 * (B1 + B2) (sum Unew = sum U - bflux); returns the first-order cells of
 * both stages, or -1 on a non-physical interior state. */
long ora_step_rk2(const ora_mesh* m, const double* U, double dt, double* Unew, double* bflux) {
    int nv = nvars(m);
    size_t n = (size_t)nblocks(m) * nv * ncell_block(m);
    double* Us = (double*)malloc(sizeof(double) * n);
    double b1[MAXV], b2[MAXV];
    long f1 = ora_stage(m, U, NULL, dt, Us, b1);
    long f2 = (f1 < 0) ? -1 : ora_stage(m, Us, U, dt, Unew, b2);
    free(Us);
    if (f1 < 0 || f2 < 0) return -1;
    if (bflux) for (int v = 0; v < nv; ++v) bflux[v] = 0.5 * (b1[v] + b2[v]);
    return f1 + f2;
}

/* nsteps steps in place, each with dt = CFL / max signal speed of the current
 * state; dts (may be NULL) receives each step's dt, bflux_total (may be NULL,
 * nvar doubles) the accumulated boundary fluxes. rk2 = 0: MUSCL-Hancock
 * steps; rk2 = 1: Heun RK2 steps. Returns 0, or -1 if a state became
 * non-physical. */
int ora_run_scheme(const ora_mesh* m, double* U, int nsteps, int rk2, double* dts, double* bflux_total) {
    int nv = nvars(m);
    size_t n = (size_t)nblocks(m) * nv * ncell_block(m);
    double* tmp = (double*)malloc(sizeof(double) * n);
    if (bflux_total) for (int v = 0; v < nv; ++v) bflux_total[v] = 0.0;
    int rc = 0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = ora_dt(m, U);
        if (!(dt > 0.0)) { rc = -1; break; }
        double bf[MAXV];
        long nf = rk2 ? ora_step_rk2(m, U, dt, tmp, bf) : ora_step(m, U, dt, tmp, bf);
        if (nf < 0) { rc = -1; break; }
        memcpy(U, tmp, sizeof(double) * n);
        if (dts) dts[s] = dt;
        if (bflux_total) for (int v = 0; v < nv; ++v) bflux_total[v] += bf[v];
    }
    free(tmp);
    return rc;
}

/* nsteps MUSCL-Hancock steps in place (ora_run_scheme with rk2 = 0). */
int ora_run(const ora_mesh* m, double* U, int nsteps, double* dts, double* bflux_total) {
    return ora_run_scheme(m, U, nsteps, 0, dts, bflux_total);
}

/* ---------------------------------------------------------------- two-level AMR
 * Block AMR with flux correction (the paper's section "Experiments": when two
 * adjacent blocks are at different refinement levels, their boundary fluxes
 * must be reconciled). The coarse level is the uniform block grid of m; the
 * blocks listed in `refined` are each covered by 2^ndim fine blocks of the
 * same cell count and half the cell width (fine block r * 2^ndim + o is child
 * o of refined[r], octant bits x | y << 1 | z << 2). Both levels advance with
 * the same dt (no subcycling). Readings:
 *   - a coarse block under fine blocks (a parent) holds the average of its
 *     children's cells (restriction) and is not advanced itself;
 *   - fine guard cells inside a fine block read it; inside an unrefined
 *     coarse block they take the value of the coarse cell that contains them
 *     (piecewise-constant prolongation); the fine level applies the boundary
 *     rule in its own index space;
 *   - coarse guard cells read the coarse level, parents included;
 *   - flux correction: a coarse leaf cell next to a refined block is updated
 *     with the average of the 2^(ndim-1) fine fluxes through its face (summed
 *     pairwise) instead of its own flux there, so every face carries one flux
 *     and the total sum_cells U dV is conserved exactly up to rounding;
 *   - dt = CFL / max over leaf cells of both levels of sum_d (|u_d| + c)/dx_d.
 * State arrays: coarse [block][var][k][j][i] over all coarse blocks (parents
 * included), fine [fine block][var][k][j][i]. */

typedef struct ora_amr_src {
    const ora_mesh* c;     /* coarse level */
    const int* child0;     /* per coarse block: its first fine block, or -1 (a leaf) */
    const double* U0;      /* coarse state (parents restricted) */
    const double* U1;      /* fine state */
} ora_amr_src;

static long cell_off(const ora_mesh* m, const int loc[3]) {
    return ((long)loc[2] * m->bs[1] + loc[1]) * m->bs[0] + loc[0];
}

/* Value of variable v at fine global cell (gi, gj, gk), indices possibly
 * outside the domain (fine-level boundary rule first). */
static double amr_value(const ora_amr_src* s, int v, int gi, int gj, int gk) {
    const ora_mesh* c = s->c;
    int nv = nvars(c), g[3] = {gi, gj, gk}, f[3], gc[3], bc[3], loc[3];
    for (int d = 0; d < 3; ++d) {
        f[d] = (d < c->ndim) ? map_index(g[d], 2 * c->nb[d] * c->bs[d], c->periodic[d]) : 0;
        gc[d] = f[d] / 2;
        if (d >= c->ndim) gc[d] = 0;
        bc[d] = gc[d] / c->bs[d];
    }
    long b = bc[0] + (long)c->nb[0] * (bc[1] + (long)c->nb[1] * bc[2]);
    if (s->child0[b] < 0) {
        for (int d = 0; d < 3; ++d) loc[d] = gc[d] % c->bs[d];
        return s->U0[(b * nv + v) * ncell_block(c) + cell_off(c, loc)];
    }
    int o = 0;
    for (int d = 0; d < c->ndim; ++d) {
        o |= ((f[d] / c->bs[d]) % 2) << d;
        loc[d] = f[d] % c->bs[d];
    }
    for (int d = c->ndim; d < 3; ++d) loc[d] = 0;
    long fb = s->child0[b] + o;
    return s->U1[(fb * nv + v) * ncell_block(c) + cell_off(c, loc)];
}

/* Parents (coarse blocks with children) <- average of their children's cells:
 * the 2^ndim fine cells (x fastest) summed pairwise, times 1/2^ndim (so equal
 * values restrict exactly). */
static void amr_restrict(const ora_mesh* c, const int* child0, const double* U1, double* U0) {
    int nv = nvars(c), nd = c->ndim;
    long nc = ncell_block(c), nblk = nblocks(c);
    double w = (nd == 3) ? 0.125 : 0.25;
    for (long b = 0; b < nblk; ++b) {
        if (child0[b] < 0) continue;
        for (int k = 0; k < c->bs[2]; ++k)
            for (int j = 0; j < c->bs[1]; ++j)
                for (int i = 0; i < c->bs[0]; ++i) {
                    int loc[3] = {i, j, k}, o = 0, fl[3];
                    for (int d = 0; d < nd; ++d) {
                        o |= ((2 * loc[d]) / c->bs[d]) << d;
                        fl[d] = (2 * loc[d]) % c->bs[d];
                    }
                    if (nd == 2) fl[2] = 0;
                    long fb = child0[b] + o;
                    for (int v = 0; v < nv; ++v) {
                        double x[8];
                        int n = 0;
                        for (int ez = 0; ez < (nd == 3 ? 2 : 1); ++ez)
                            for (int ey = 0; ey < 2; ++ey)
                                for (int ex = 0; ex < 2; ++ex) {
                                    int q[3] = {fl[0] + ex, fl[1] + ey, fl[2] + ez};
                                    x[n++] = U1[(fb * nv + v) * nc + cell_off(c, q)];
                                }
                        double s = (x[0] + x[1]) + (x[2] + x[3]);
                        if (nd == 3) s = s + ((x[4] + x[5]) + (x[6] + x[7]));
                        U0[(b * nv + v) * nc + cell_off(c, loc)] = w * s;
                    }
                }
    }
}

static int* amr_children(const ora_mesh* c, const int* refined, int nref) {
    long nblk = nblocks(c);
    int* child0 = (int*)malloc(sizeof(int) * (size_t)nblk);
    for (long b = 0; b < nblk; ++b) child0[b] = -1;
    for (int r = 0; r < nref; ++r) child0[refined[r]] = r << c->ndim;
    return child0;
}

/* The fine level as a uniform mesh of twice as many blocks per axis (used
 * for cell widths, block coordinates and its boundary rule). */
static ora_mesh amr_fine_mesh(const ora_mesh* c) {
    ora_mesh f = *c;
    for (int d = 0; d < c->ndim; ++d) f.nb[d] = 2 * c->nb[d];
    return f;
}

/* Largest signal speed over the leaf cells of both levels; -1 if a leaf cell
 * is non-physical. */
double ora_amr_max_signal_speed(const ora_mesh* c, const int* refined, int nref, const double* U0,
                                const double* U1) {
    int nv = nvars(c), nch = 1 << c->ndim;
    int* child0 = amr_children(c, refined, nref);
    ora_mesh f = amr_fine_mesh(c);
    double idxc[3], idxf[3], smax = 0.0;
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
        idxc[d] = 1.0 / cell_width(c, d);
        idxf[d] = 1.0 / cell_width(&f, d);
    }
    long nc = ncell_block(c), nblk = nblocks(c), nfine = (long)nref * nch;
    for (long b = 0; b < nblk + nfine; ++b) {
        int fine = b >= nblk;
        if (!fine && child0[b] >= 0) continue;
        const double* U = fine ? U1 : U0;
        long bb = fine ? b - nblk : b;
        for (long cc = 0; cc < nc; ++cc) {
            double Uc[MAXV], W[MAXV], r;
            for (int v = 0; v < nv; ++v) Uc[v] = U[(bb * nv + v) * nc + cc];
            prim_from_cons(c->ndim, c->gamma, Uc, W, &r);
            if (!(W[0] > 0.0) || !(W[nv - 1] > 0.0)) bad = 1;
            double s = cell_signal_speed(c, Uc, fine ? idxf : idxc);
            if (s > smax) smax = s;
        }
    }
    free(child0);
    return bad ? -1.0 : smax;
}

double ora_amr_dt(const ora_mesh* c, const int* refined, int nref, const double* U0, const double* U1) {
    double s = ora_amr_max_signal_speed(c, refined, nref, U0, U1);
    if (!(s > 0.0)) return -1.0;
    return c->cfl / s;
}

/* One two-level MUSCL-Hancock step with dt: parents restricted from U1, every
 * leaf block of both levels advanced (fine guards by the rule above), then
 * the flux correction at coarse-fine faces, then the parents of U0new
 * restricted from U1new. Returns the first-order cells, or -1 on a
 * non-physical leaf state. */
long ora_amr_step(const ora_mesh* c, const int* refined, int nref, const double* U0, const double* U1, double dt,
                  double* U0new, double* U1new) {
    int nv = nvars(c), nd = c->ndim, nch = 1 << nd;
    long nc = ncell_block(c), nblk = nblocks(c), nfine = (long)nref * nch;
    int* child0 = amr_children(c, refined, nref);
    ora_mesh f = amr_fine_mesh(c);
    long fsz = face_stride(c), regsz = 6 * MAXV * fsz;
    double* P = (double*)malloc(sizeof(double) * (size_t)(nblk * nv * nc));
    memcpy(P, U0, sizeof(double) * (size_t)(nblk * nv * nc));
    amr_restrict(c, child0, U1, P);
    memcpy(U0new, P, sizeof(double) * (size_t)(nblk * nv * nc));
    double* regc = (double*)calloc((size_t)(nblk * regsz), sizeof(double));
    double* regf = (double*)calloc((size_t)(nfine > 0 ? nfine * regsz : 1), sizeof(double));
    ora_amr_src src = {c, child0, P, U1};
    long nfirst = 0, nbad = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads) reduction(+ : nfirst, nbad)
#endif
    {
        ora_work w;
        for (int d = 0; d < 3; ++d) {
            w.off[d] = (d < nd) ? G : 0;
            w.p[d] = c->bs[d] + 2 * w.off[d];
        }
        long np = (long)w.p[0] * w.p[1] * w.p[2];
        w.U = (double*)malloc(sizeof(double) * np * MAXV);
        w.W = (double*)malloc(sizeof(double) * np * MAXV);
        w.R = (double*)malloc(sizeof(double) * np);
        w.FS = (double*)malloc(sizeof(double) * np * 3 * 2 * MAXV);
        w.first = (int*)calloc((size_t)np, sizeof(int));
        double bf[MAXV];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long b = 0; b < nblk + nfine; ++b) {
            for (int v = 0; v < MAXV; ++v) bf[v] = 0.0;
            if (b < nblk) {                       /* a coarse leaf */
                if (child0[b] >= 0) continue;
                w.amr = NULL;
                w.reg = regc + b * regsz;
                w.out_b = -1;
                advance_block(c, P, NULL, 1, dt, b, U0new, bf, &nfirst, &nbad, &w);
            } else {                              /* a fine block: its coordinates on the fine level */
                long fb = b - nblk;
                int pr = refined[fb >> nd], o = (int)(fb & (nch - 1));
                int pc[3] = {pr % c->nb[0], (pr / c->nb[0]) % c->nb[1], pr / (c->nb[0] * c->nb[1])}, fc[3];
                for (int d = 0; d < 3; ++d) fc[d] = (d < nd) ? 2 * pc[d] + ((o >> d) & 1) : 0;
                long ub = fc[0] + (long)f.nb[0] * (fc[1] + (long)f.nb[1] * fc[2]);
                w.amr = &src;
                w.reg = regf + fb * regsz;
                w.out_b = fb;
                advance_block(&f, U1, NULL, 1, dt, ub, U1new, bf, &nfirst, &nbad, &w);
            }
        }
        free(w.U); free(w.W); free(w.R); free(w.FS); free(w.first);
    }
    /* flux correction at the faces between coarse leaves and refined blocks */
    for (long b = 0; b < nblk; ++b) {
        if (child0[b] >= 0) continue;
        int bc[3] = {(int)(b % c->nb[0]), (int)((b / c->nb[0]) % c->nb[1]), (int)(b / ((long)c->nb[0] * c->nb[1]))};
        for (int d = 0; d < nd; ++d)
            for (int side = 0; side < 2; ++side) {
                int nbc[3] = {bc[0], bc[1], bc[2]};
                nbc[d] += side ? 1 : -1;
                if (nbc[d] < 0 || nbc[d] >= c->nb[d]) {
                    if (!c->periodic[d]) continue;
                    nbc[d] = (nbc[d] + c->nb[d]) % c->nb[d];
                }
                long N = nbc[0] + (long)c->nb[0] * (nbc[1] + (long)c->nb[1] * nbc[2]);
                if (child0[N] < 0) continue;
                int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
                double cdc = dt * (1.0 / cell_width(c, d));
                for (int t2 = 0; t2 < c->bs[a2]; ++t2)
                    for (int t1 = 0; t1 < c->bs[a1]; ++t1) {
                        int loc[3];
                        loc[d] = side ? c->bs[d] - 1 : 0;
                        loc[a1] = t1;
                        loc[a2] = t2;
                        long t = face_cell(c, d, loc);
                        /* the children of N on the near side, and their face cells */
                        int s1 = (2 * t1) / c->bs[a1], s2 = (a2 < nd) ? (2 * t2) / c->bs[a2] : 0;
                        int o = ((side ? 0 : 1) << d) | (s1 << a1) | (s2 << a2);
                        long fb = child0[N] + o;
                        const double* rf = regf + fb * regsz + ((2 * d + (side ? 0 : 1)) * MAXV) * fsz;
                        const double* rc = regc + b * regsz + ((2 * d + side) * MAXV) * fsz;
                        for (int v = 0; v < nv; ++v) {
                            double avg;
                            int fl[3];
                            fl[d] = 0;
                            fl[a1] = 2 * t1 - s1 * c->bs[a1];
                            fl[a2] = (a2 < nd) ? 2 * t2 - s2 * c->bs[a2] : 0;
                            if (nd == 3) {
                                int q00[3] = {fl[0], fl[1], fl[2]}, q10[3], q01[3], q11[3];
                                for (int e = 0; e < 3; ++e) { q10[e] = q00[e]; q01[e] = q00[e]; q11[e] = q00[e]; }
                                q10[a1] += 1; q01[a2] += 1; q11[a1] += 1; q11[a2] += 1;
                                avg = 0.25 * ((rf[v * fsz + face_cell(c, d, q00)] + rf[v * fsz + face_cell(c, d, q10)]) +
                                              (rf[v * fsz + face_cell(c, d, q01)] + rf[v * fsz + face_cell(c, d, q11)]));
                            } else {
                                int q0[3] = {fl[0], fl[1], 0}, q1[3] = {fl[0], fl[1], 0};
                                q1[a1] += 1;
                                avg = 0.5 * (rf[v * fsz + face_cell(c, d, q0)] + rf[v * fsz + face_cell(c, d, q1)]);
                            }
                            double corr = cdc * (rc[v * fsz + t] - avg);
                            long oi = (b * nv + v) * nc + cell_off(c, loc);
                            U0new[oi] = side ? (U0new[oi] + corr) : (U0new[oi] - corr);
                        }
                    }
            }
    }
    amr_restrict(c, child0, U1new, U0new);
    free(P); free(regc); free(regf); free(child0);
    return nbad ? -1 : nfirst;
}
