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
} ora_work;

static long pidx(const ora_work* w, int i, int j, int k) {
    return ((long)(k + w->off[2]) * w->p[1] + (j + w->off[1])) * w->p[0] + (i + w->off[0]);
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
                    w->U[v * np + pidx(w, i, j, k)] = global_value(m, U, v, gi, gj, gk);
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
                    if (!m->periodic[d]) {
                        if (bxyz[d] == 0 && loc[d] == 0)
                            for (int v = 0; v < nv; ++v) bflux[v] -= cd[d] * Flo[v];
                        if (bxyz[d] == m->nb[d] - 1 && loc[d] == m->bs[d] - 1)
                            for (int v = 0; v < nv; ++v) bflux[v] += cd[d] * Fhi[v];
                    }
                }
                long co = ((long)k * m->bs[1] + j) * m->bs[0] + i;
                for (int v = 0; v < nv; ++v) {
                    long o = (b * nv + v) * ncell_block(m) + co;
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
