/*
 * FP64 reference stepper for the fictitious-wave Maxwell system -- TEST
 * INFRASTRUCTURE ONLY.  Nothing in the product path may call this file; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 *
 * What it computes (paper Sec. 2):
 *   mu  dH'/dt' = -curl E' + M'         (Eq. 4, first row, M' = 0 here)
 *   eps dE'/dt' =  curl H' - J'         (Eq. 4, second row)
 * by the leap-frog staggered-grid (Yee) scheme on a tensor-product grid with
 * non-uniform spacing, unsplit convolutional PML (Komatitsch & Martin 2007)
 * on the outer faces, point injection of J' and point sampling of E', and
 * the on-the-fly damped transform of Eq. 6:
 *   u(x, w_k) = sum_{n=0}^{nt-1} u(x, n dt) exp((-1 + i) sqrt(w_k w0) n dt).
 *
 * Layout: every field component lives on the (nx+1)(ny+1)(nz+1) node lattice,
 *   index (k*(ny+1) + j)*(nx+1) + i, with the Yee offsets implied:
 *   Ex(i,j,k) at (i+1/2, j, k)        Hx(i,j,k) at (i, j+1/2, k+1/2)
 *   Ey(i,j,k) at (i, j+1/2, k)        Hy(i,j,k) at (i+1/2, j, k+1/2)
 *   Ez(i,j,k) at (i, j, k+1/2)        Hz(i,j,k) at (i+1/2, j+1/2, k)
 * Entries outside a component's lattice stay zero.  Tangential E on the
 * outer boundary is never updated (perfect conductor behind the CPML).
 *
 * Every array is full-size and every loop visits every point: slow on
 * purpose, so that each line can be checked against the equations.
 *
 * Spatial order (Sec. 2 uses high-order differences on the non-uniform grid):
 * order 2 is the two-point Yee difference.  Order 4 takes, at each half node
 * p, the four-point weights wh[p][0..3] on the nodes p-1 .. p+2 (H update),
 * and at each node q the weights wn[q][0..3] on the half nodes q-2 .. q+1
 * (E update); the tables come from the caller, terms outside the lattice are
 * skipped (their weights are zero).
 */
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the parallel loops (timing runs use 1 and all host cores). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int nx, ny, nz;
    /* 1/h at half nodes (len n) and 1/h~ at nodes (len n+1), per axis */
    const double *ihx_h, *ihx_n, *ihy_h, *ihy_n, *ihz_h, *ihz_n;
    /* CPML recursion coefficients psi <- b psi + a d(u), at half nodes and nodes */
    const double *bx_h, *ax_h, *bx_n, *ax_n;
    const double *by_h, *ay_h, *by_n, *ay_n;
    const double *bz_h, *az_h, *bz_n, *az_n;
    double cH;          /* dt / mu0 */
    const double *cE;   /* [3][N] dt / eps on each E edge */
    int order;          /* 2 or 4 */
    /* order 4: weights at half nodes [n][4] and at nodes [n+1][4], per axis */
    const double *wx_h, *wx_n, *wy_h, *wy_n, *wz_h, *wz_n;
} orc_model;

/* d/da of a node-located field at half node p along an axis of n cells;
 * F + at is the field at node p, s the stride along the axis. */
static double d_half(const double *F, size_t at, size_t s, int p, int n, int order, const double *ih,
                     const double *wh)
{
    if (order != 4) return (F[at + s] - F[at]) * ih[p];
    double d = 0.0;
    for (int o = 0; o < 4; ++o) {
        const int q = p - 1 + o;
        if (q >= 0 && q <= n) d += wh[4 * p + o] * F[at + (size_t)(o - 1) * s];
    }
    return d;
}

/* d/da of a half-node-located field at node p; F + at is the field at half node p. */
static double d_node(const double *F, size_t at, size_t s, int p, int n, int order, const double *ih,
                     const double *wn)
{
    if (order != 4) return (F[at] - F[at - s]) * ih[p];
    double d = 0.0;
    for (int o = 0; o < 4; ++o) {
        const int q = p - 2 + o;
        if (q >= 0 && q <= n - 1) d += wn[4 * p + o] * F[at + (size_t)(o - 2) * s];
    }
    return d;
}

typedef struct {
    /* point injection: J'_edge(t_{n+1/2}) = w * series[e][n] (w already holds 1/dV) */
    int n_inj;
    const int *comp, *i, *j, *k, *emitter;
    const double *w;
    const double *series;   /* [n_emit][nt] */
    /* point sampling of E at t_n: trace[r][n] = sum_taps w * E_comp */
    int n_tap, n_rec;
    const int *tcomp, *ti, *tj, *tk, *trec;
    const double *tw;
    double *trace;          /* [n_rec][nt] or NULL */
    /* volumetric transform of E at t_n */
    int n_freq;
    const double *dft_re, *dft_im;  /* [nt][n_freq] */
    double *vol_re, *vol_im;        /* [3][n_freq][N] or NULL */
    int nt;
} orc_io;

#define AT(a, i, j, k) (a)[((size_t)(k) * (size_t)(ny + 1) + (size_t)(j)) * (size_t)(nx + 1) + (size_t)(i)]
#define IX(i, j, k) (((size_t)(k) * (size_t)(ny + 1) + (size_t)(j)) * (size_t)(nx + 1) + (size_t)(i))

/* fields: [6][N] = Ex,Ey,Ez,Hx,Hy,Hz.  psi: [12][N]. Runs steps n0..n1-1. */
int orc_run(const orc_model *m, const orc_io *io, double *fields, double *psi, int n0, int n1)
{
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    const size_t N = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    double *Ex = fields, *Ey = fields + N, *Ez = fields + 2 * N;
    double *Hx = fields + 3 * N, *Hy = fields + 4 * N, *Hz = fields + 5 * N;
    /* psi for the H update (derivatives of E) and for the E update (derivatives of H) */
    double *p_hx_y = psi, *p_hx_z = psi + N, *p_hy_z = psi + 2 * N;
    double *p_hy_x = psi + 3 * N, *p_hz_x = psi + 4 * N, *p_hz_y = psi + 5 * N;
    double *p_ex_y = psi + 6 * N, *p_ex_z = psi + 7 * N, *p_ey_z = psi + 8 * N;
    double *p_ey_x = psi + 9 * N, *p_ez_x = psi + 10 * N, *p_ez_y = psi + 11 * N;
    const double *cEx = m->cE, *cEy = m->cE + N, *cEz = m->cE + 2 * N;
    const double cH = m->cH;
    const int od = m->order;
    const size_t sx = 1, sy = (size_t)(nx + 1), sz = (size_t)(nx + 1) * (size_t)(ny + 1);

    for (int n = n0; n < n1; ++n) {
        /* ---- sample E^n at the receivers ---- */
        if (io->trace) {
            for (int p = 0; p < io->n_tap; ++p) {
                const double *Ec = fields + (size_t)io->tcomp[p] * N;
                io->trace[(size_t)io->trec[p] * io->nt + n] += io->tw[p] * AT(Ec, io->ti[p], io->tj[p], io->tk[p]);
            }
        }
        /* ---- volumetric damped transform of E^n (Eq. 6) ---- */
        if (io->vol_re) {
            for (int c = 0; c < 3; ++c) {
                const double *Ec = fields + (size_t)c * N;
                for (int f = 0; f < io->n_freq; ++f) {
                    const double wr = io->dft_re[(size_t)n * io->n_freq + f];
                    const double wi = io->dft_im[(size_t)n * io->n_freq + f];
                    double *vr = io->vol_re + ((size_t)c * io->n_freq + f) * N;
                    double *vi = io->vol_im + ((size_t)c * io->n_freq + f) * N;
                    #pragma omp parallel for schedule(static)
                    for (long q = 0; q < (long)N; ++q) {
                        vr[q] += Ec[q] * wr;
                        vi[q] += Ec[q] * wi;
                    }
                }
            }
        }

        /* ---- H^{n-1/2} -> H^{n+1/2}:  H -= dt/mu0 * curl E^n ---- */
        #pragma omp parallel for schedule(static)
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    if (j < ny && k < nz) {             /* Hx at (i, j+1/2, k+1/2) */
                        double dEz_dy = d_half(Ez, IX(i, j, k), sy, j, ny, od, m->ihy_h, m->wy_h);
                        double dEy_dz = d_half(Ey, IX(i, j, k), sz, k, nz, od, m->ihz_h, m->wz_h);
                        AT(p_hx_y, i, j, k) = m->by_h[j] * AT(p_hx_y, i, j, k) + m->ay_h[j] * dEz_dy;
                        AT(p_hx_z, i, j, k) = m->bz_h[k] * AT(p_hx_z, i, j, k) + m->az_h[k] * dEy_dz;
                        AT(Hx, i, j, k) -= cH * ((dEz_dy + AT(p_hx_y, i, j, k)) - (dEy_dz + AT(p_hx_z, i, j, k)));
                    }
                    if (i < nx && k < nz) {             /* Hy at (i+1/2, j, k+1/2) */
                        double dEx_dz = d_half(Ex, IX(i, j, k), sz, k, nz, od, m->ihz_h, m->wz_h);
                        double dEz_dx = d_half(Ez, IX(i, j, k), sx, i, nx, od, m->ihx_h, m->wx_h);
                        AT(p_hy_z, i, j, k) = m->bz_h[k] * AT(p_hy_z, i, j, k) + m->az_h[k] * dEx_dz;
                        AT(p_hy_x, i, j, k) = m->bx_h[i] * AT(p_hy_x, i, j, k) + m->ax_h[i] * dEz_dx;
                        AT(Hy, i, j, k) -= cH * ((dEx_dz + AT(p_hy_z, i, j, k)) - (dEz_dx + AT(p_hy_x, i, j, k)));
                    }
                    if (i < nx && j < ny) {             /* Hz at (i+1/2, j+1/2, k) */
                        double dEy_dx = d_half(Ey, IX(i, j, k), sx, i, nx, od, m->ihx_h, m->wx_h);
                        double dEx_dy = d_half(Ex, IX(i, j, k), sy, j, ny, od, m->ihy_h, m->wy_h);
                        AT(p_hz_x, i, j, k) = m->bx_h[i] * AT(p_hz_x, i, j, k) + m->ax_h[i] * dEy_dx;
                        AT(p_hz_y, i, j, k) = m->by_h[j] * AT(p_hz_y, i, j, k) + m->ay_h[j] * dEx_dy;
                        AT(Hz, i, j, k) -= cH * ((dEy_dx + AT(p_hz_x, i, j, k)) - (dEx_dy + AT(p_hz_y, i, j, k)));
                    }
                }

        /* ---- E^n -> E^{n+1}:  E += dt/eps * (curl H^{n+1/2} - J'^{n+1/2}) ---- */
        #pragma omp parallel for schedule(static)
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    if (i < nx && j >= 1 && j < ny && k >= 1 && k < nz) {   /* Ex */
                        double dHz_dy = d_node(Hz, IX(i, j, k), sy, j, ny, od, m->ihy_n, m->wy_n);
                        double dHy_dz = d_node(Hy, IX(i, j, k), sz, k, nz, od, m->ihz_n, m->wz_n);
                        AT(p_ex_y, i, j, k) = m->by_n[j] * AT(p_ex_y, i, j, k) + m->ay_n[j] * dHz_dy;
                        AT(p_ex_z, i, j, k) = m->bz_n[k] * AT(p_ex_z, i, j, k) + m->az_n[k] * dHy_dz;
                        AT(Ex, i, j, k) += AT(cEx, i, j, k) * ((dHz_dy + AT(p_ex_y, i, j, k)) - (dHy_dz + AT(p_ex_z, i, j, k)));
                    }
                    if (j < ny && i >= 1 && i < nx && k >= 1 && k < nz) {   /* Ey */
                        double dHx_dz = d_node(Hx, IX(i, j, k), sz, k, nz, od, m->ihz_n, m->wz_n);
                        double dHz_dx = d_node(Hz, IX(i, j, k), sx, i, nx, od, m->ihx_n, m->wx_n);
                        AT(p_ey_z, i, j, k) = m->bz_n[k] * AT(p_ey_z, i, j, k) + m->az_n[k] * dHx_dz;
                        AT(p_ey_x, i, j, k) = m->bx_n[i] * AT(p_ey_x, i, j, k) + m->ax_n[i] * dHz_dx;
                        AT(Ey, i, j, k) += AT(cEy, i, j, k) * ((dHx_dz + AT(p_ey_z, i, j, k)) - (dHz_dx + AT(p_ey_x, i, j, k)));
                    }
                    if (k < nz && i >= 1 && i < nx && j >= 1 && j < ny) {   /* Ez */
                        double dHy_dx = d_node(Hy, IX(i, j, k), sx, i, nx, od, m->ihx_n, m->wx_n);
                        double dHx_dy = d_node(Hx, IX(i, j, k), sy, j, ny, od, m->ihy_n, m->wy_n);
                        AT(p_ez_x, i, j, k) = m->bx_n[i] * AT(p_ez_x, i, j, k) + m->ax_n[i] * dHy_dx;
                        AT(p_ez_y, i, j, k) = m->by_n[j] * AT(p_ez_y, i, j, k) + m->ay_n[j] * dHx_dy;
                        AT(Ez, i, j, k) += AT(cEz, i, j, k) * ((dHy_dx + AT(p_ez_x, i, j, k)) - (dHx_dy + AT(p_ez_y, i, j, k)));
                    }
                }
        /* source term: E -= dt/eps * J'^{n+1/2} */
        for (int p = 0; p < io->n_inj; ++p) {
            double *Ec = fields + (size_t)io->comp[p] * N;
            const double *cc = m->cE + (size_t)io->comp[p] * N;
            const double amp = io->w[p] * io->series[(size_t)io->emitter[p] * io->nt + n];
            AT(Ec, io->i[p], io->j[p], io->k[p]) -= AT(cc, io->i[p], io->j[p], io->k[p]) * amp;
        }
    }
    return 0;
}
