/*
 * oracle4pcf.c -- plain, slow, FP64 CPU oracle for the multipole estimator of the shear
 * 4PCF of Porth et al. (arXiv:2509.07974).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU legs of
 * bench.py to check the CUDA library; it shares no code with it.
 *
 * Every step follows the paper in its order and notation:
 *   - shear projection gamma(theta; zeta) = -gamma_c exp(-2 i zeta)     (Eq. gammatx_def)
 *   - the x-projection zeta_0 = (phi_1+phi_3)/2, zeta_k = phi_k         (Eq. xprojection)
 *   - per-centre multipoles G_n(theta_i, Theta) = sum_j w_j gamma_c,j e^{i n phi_ij} over
 *     neighbours in the radial bin, and W_n likewise with w_j        (Eq. 4PCFUpsilon0)
 *   - Upsilon_{mu,n} as the products printed for mu = 0..7 and N_n (Eq. Nnmultipoles)
 *   - multiple-counting corrections of Table tab:4PCFMCCorr (App. A.1)
 *   - multipole -> real space (Eq. Multipole2RealConversion), Gamma = Upsilon / N
 *     (Eq. 4PCF_quadrupletestimator), bin-averaged as in Eq. Gamma0_binned
 *   - fourth-order aperture measures (Eq. 4PCF2M4) for the filter of Eq. CrittendenQ, the
 *     correlator order of Eq. M4Ordering and the component order of
 *     Eq. 4PCF_rawcomponents.
 * Floating point: compile with -ffp-contract=off so that dx*dx + dy*dy is evaluated as two
 * rounded products and one rounded sum (the radial-bin decision is then reproducible).
 */
#include "oracle4pcf.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define NCOMP 9 /* eight natural components + normalisation */

/* ------------------------------------------------------------------------------------ */
/* Radial binning: bin b holds separations with edges[b]^2 <= r^2 < edges[b+1]^2.        */
/* ------------------------------------------------------------------------------------ */
static int radial_bin(double r2, const double* e2, int nb) {
  for (int b = 0; b < nb; ++b)
    if (e2[b] <= r2 && r2 < e2[b + 1]) return b;
  return -1;
}

static int check_edges(const double* edges, int nb) {
  if (nb < 1 || !(edges[0] > 0.0)) return -1;
  for (int b = 0; b < nb; ++b)
    if (!(edges[b + 1] > edges[b])) return -1;
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* A plain uniform cell list of cell size edges[nb] (the largest separation), so that all  */
/* partners of a galaxy lie in the 3x3 block of cells around it.                          */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double x0, y0, cs;
  int64_t nx, ny;
  int64_t* start; /* [nx*ny+1] */
  int64_t* items; /* galaxy indices, grouped by cell */
} cell_list;

static void cell_of(const cell_list* cl, double x, double y, int64_t* cx, int64_t* cy) {
  int64_t ix = (int64_t)floor((x - cl->x0) / cl->cs);
  int64_t iy = (int64_t)floor((y - cl->y0) / cl->cs);
  if (ix < 0) ix = 0;
  if (iy < 0) iy = 0;
  if (ix >= cl->nx) ix = cl->nx - 1;
  if (iy >= cl->ny) iy = cl->ny - 1;
  *cx = ix;
  *cy = iy;
}

static int cell_list_build(cell_list* cl, int64_t n, const double* pos, double rmax) {
  double xmin = pos[0], xmax = pos[0], ymin = pos[1], ymax = pos[1];
  for (int64_t i = 1; i < n; ++i) {
    if (pos[2 * i] < xmin) xmin = pos[2 * i];
    if (pos[2 * i] > xmax) xmax = pos[2 * i];
    if (pos[2 * i + 1] < ymin) ymin = pos[2 * i + 1];
    if (pos[2 * i + 1] > ymax) ymax = pos[2 * i + 1];
  }
  cl->x0 = xmin;
  cl->y0 = ymin;
  /* cells no smaller than the largest separation (and at most ~4000 per axis) */
  double cs = rmax;
  if ((xmax - xmin) / 4000.0 > cs) cs = (xmax - xmin) / 4000.0;
  if ((ymax - ymin) / 4000.0 > cs) cs = (ymax - ymin) / 4000.0;
  cl->cs = cs;
  cl->nx = (int64_t)floor((xmax - xmin) / cs) + 1;
  cl->ny = (int64_t)floor((ymax - ymin) / cs) + 1;
  int64_t nc = cl->nx * cl->ny;
  cl->start = (int64_t*)calloc((size_t)(nc + 1), sizeof(int64_t));
  cl->items = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc((size_t)nc, sizeof(int64_t));
  if (!cl->start || !cl->items || !fill) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx, cy;
    cell_of(cl, pos[2 * i], pos[2 * i + 1], &cx, &cy);
    cl->start[cy * cl->nx + cx + 1]++;
  }
  for (int64_t c = 0; c < nc; ++c) cl->start[c + 1] += cl->start[c];
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx, cy;
    cell_of(cl, pos[2 * i], pos[2 * i + 1], &cx, &cy);
    int64_t c = cy * cl->nx + cx;
    cl->items[cl->start[c] + fill[c]++] = i;
  }
  free(fill);
  return 0;
}

static void cell_list_free(cell_list* cl) {
  free(cl->start);
  free(cl->items);
}

/* ------------------------------------------------------------------------------------ */
/* Per-centre multipoles (step A of App. A.2).  For centre i and radial bin b:            */
/*   G_n   = sum_j x_j e^{i n phi_ij},   x_j = w_j gamma_c,j       n in [-2N-3, 2N-1]      */
/*   W_n   = sum_j w_j e^{i n phi_ij}                              n in [-2N,   2N  ]      */
/* and the quantities that Table tab:4PCFMCCorr multiplies with g:                        */
/*   XX_n  = sum_j x_j^2 e^{i n phi}        n in [-2N-6, 2N-2]                             */
/*   XA_n  = sum_j |x_j|^2 e^{i n phi}      n in [-2N-2, 2N+2]                             */
/*   WW_n  = sum_j w_j^2 e^{i n phi}        n in [-2N,   2N  ]                             */
/*   XXX_{-8}, XXX_{-4} (x^3), XXC_{-4}, XXC_0 (x^2 x^*), WWW_0 (w^3)                      */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  int N, nb;
  int oG, nG, oW, nW, oXX, nXX, oXA, nXA;
  size_t per_centre; /* complex values per centre */
} mp_dims;

static mp_dims make_dims(int N, int nb) {
  mp_dims d;
  d.N = N;
  d.nb = nb;
  d.oG = 2 * N + 3;
  d.nG = 4 * N + 3;
  d.oW = 2 * N;
  d.nW = 4 * N + 1;
  d.oXX = 2 * N + 6;
  d.nXX = 4 * N + 5;
  d.oXA = 2 * N + 2;
  d.nXA = 4 * N + 5;
  /* G, W, XX, XA, WW (same range as W), 5 triple terms, per bin; plus x_i and w_i */
  d.per_centre = (size_t)nb * (size_t)(d.nG + d.nW + d.nXX + d.nXA + d.nW + 5) + 2;
  return d;
}

typedef struct {
  const mp_dims* d;
  cplx* base;
} centre_mp;

static cplx* mp_G(centre_mp c) { return c.base; }
static cplx* mp_W(centre_mp c) { return c.base + (size_t)c.d->nb * c.d->nG; }
static cplx* mp_XX(centre_mp c) { return mp_W(c) + (size_t)c.d->nb * c.d->nW; }
static cplx* mp_XA(centre_mp c) { return mp_XX(c) + (size_t)c.d->nb * c.d->nXX; }
static cplx* mp_WW(centre_mp c) { return mp_XA(c) + (size_t)c.d->nb * c.d->nXA; }
static cplx* mp_TR(centre_mp c) { return mp_WW(c) + (size_t)c.d->nb * c.d->nW; }
static cplx* mp_XW(centre_mp c) { return mp_TR(c) + (size_t)c.d->nb * 5; }

/* accessors with the paper's index n */
#define G(b, n) (mp_G(c)[(size_t)(b) * c.d->nG + (size_t)((n) + c.d->oG)])
#define W(b, n) (mp_W(c)[(size_t)(b) * c.d->nW + (size_t)((n) + c.d->oW)])
#define XX(b, n) (mp_XX(c)[(size_t)(b) * c.d->nXX + (size_t)((n) + c.d->oXX)])
#define XA(b, n) (mp_XA(c)[(size_t)(b) * c.d->nXA + (size_t)((n) + c.d->oXA)])
#define WW(b, n) (mp_WW(c)[(size_t)(b) * c.d->nW + (size_t)((n) + c.d->oW)])
#define XXX_M8(b) (mp_TR(c)[(size_t)(b) * 5 + 0])
#define XXX_M4(b) (mp_TR(c)[(size_t)(b) * 5 + 1])
#define XXC_M4(b) (mp_TR(c)[(size_t)(b) * 5 + 2])
#define XXC_0(b) (mp_TR(c)[(size_t)(b) * 5 + 3])
#define WWW_0(b) (mp_TR(c)[(size_t)(b) * 5 + 4])
#define XI (mp_XW(c)[0])
#define WI (mp_XW(c)[1])

static void centre_multipoles(int64_t i, int64_t n, const double* pos, const double* shear,
                              const double* w, const double* e2, const cell_list* cl,
                              centre_mp c) {
  const mp_dims* d = c.d;
  const int N = d->N, nb = d->nb;
  memset(c.base, 0, d->per_centre * sizeof(cplx));
  XI = w[i] * (shear[2 * i] + I * shear[2 * i + 1]);
  WI = w[i];
  int64_t cx, cy;
  cell_of(cl, pos[2 * i], pos[2 * i + 1], &cx, &cy);
  for (int64_t yy = cy - 1; yy <= cy + 1; ++yy) {
    if (yy < 0 || yy >= cl->ny) continue;
    for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
      if (xx < 0 || xx >= cl->nx) continue;
      int64_t cc = yy * cl->nx + xx;
      for (int64_t t = cl->start[cc]; t < cl->start[cc + 1]; ++t) {
        int64_t j = cl->items[t];
        if (j == i) continue;
        double dx = pos[2 * j] - pos[2 * i];
        double dy = pos[2 * j + 1] - pos[2 * i + 1];
        double r2 = dx * dx + dy * dy;
        int b = radial_bin(r2, e2, nb);
        if (b < 0) continue;
        double phi = atan2(dy, dx); /* polar angle of theta_j - theta_i */
        cplx xj = w[j] * (shear[2 * j] + I * shear[2 * j + 1]);
        cplx xx2 = xj * xj, xa = xj * conj(xj), ww = w[j] * w[j];
        for (int m = -2 * N - 6; m <= 2 * N + 2; ++m) {
          cplx e = cexp(I * (double)m * phi);
          if (m >= -2 * N - 3 && m <= 2 * N - 1) G(b, m) += xj * e;
          if (m >= -2 * N && m <= 2 * N) {
            W(b, m) += w[j] * e;
            WW(b, m) += ww * e;
          }
          if (m <= 2 * N - 2) XX(b, m) += xx2 * e;
          if (m >= -2 * N - 2) XA(b, m) += xa * e;
        }
        XXX_M8(b) += xj * xj * xj * cexp(-8.0 * I * phi);
        XXX_M4(b) += xj * xj * xj * cexp(-4.0 * I * phi);
        XXC_M4(b) += xj * xj * conj(xj) * cexp(-4.0 * I * phi);
        XXC_0(b) += xj * xj * conj(xj);
        WWW_0(b) += w[j] * w[j] * w[j];
      }
    }
  }
}

/* Upsilon_{mu,n}(Theta1,Theta2,Theta3) contribution of one centre, as printed after
 * Eq. 4PCFUpsilon0 (mu = 0..7) and in Eq. Nnmultipoles (mu = 8). */
static cplx upsilon_term(int mu, int n2, int n3, int b1, int b2, int b3, centre_mp c) {
  const int s = n2 + n3;
  switch (mu) {
    case 0: return XI * G(b1, s - 3) * G(b2, -(n2 + 2)) * G(b3, -(n3 + 3));
    case 1: return conj(XI) * G(b1, s - 1) * G(b2, -(n2 + 2)) * G(b3, -(n3 + 1));
    case 2: return XI * conj(G(b1, -(s + 1))) * G(b2, -(n2 + 2)) * G(b3, -(n3 + 3));
    case 3: return XI * G(b1, s - 3) * conj(G(b2, n2 - 2)) * G(b3, -(n3 + 3));
    case 4: return XI * G(b1, s - 3) * G(b2, -(n2 + 2)) * conj(G(b3, n3 - 1));
    case 5: return conj(XI) * conj(G(b1, -(s + 3))) * G(b2, -(n2 + 2)) * G(b3, -(n3 + 1));
    case 6: return conj(XI) * G(b1, s - 1) * conj(G(b2, n2 - 2)) * G(b3, -(n3 + 1));
    case 7: return conj(XI) * G(b1, s - 1) * G(b2, -(n2 + 2)) * conj(G(b3, n3 - 3));
    default: return WI * W(b1, s) * W(b2, -n2) * W(b3, -n3);
  }
}

/* Double-counting terms of Table tab:4PCFMCCorr for one centre.  Each entry is the
 * centre's x (or x^*, or w) times the merged-slot quantity g of the table times the
 * multipole of the slot that is not merged. */
static cplx corr_t1_eq_t2(int mu, int n2, int n3, int b12, int b3, centre_mp c) {
  (void)n2;
  switch (mu) {
    case 0: return XI * XX(b12, n3 - 5) * G(b3, -(n3 + 3));
    case 1: return conj(XI) * XX(b12, n3 - 3) * G(b3, -(n3 + 1));
    case 2: return XI * XA(b12, n3 - 1) * G(b3, -(n3 + 3));
    case 3: return XI * XA(b12, n3 - 1) * G(b3, -(n3 + 3));
    case 4: return XI * XX(b12, n3 - 5) * conj(G(b3, n3 - 1));
    case 5: return conj(XI) * XA(b12, n3 + 1) * G(b3, -(n3 + 1));
    case 6: return conj(XI) * XA(b12, n3 + 1) * G(b3, -(n3 + 1));
    case 7: return conj(XI) * XX(b12, n3 - 3) * conj(G(b3, n3 - 3));
    default: return WI * WW(b12, n3) * W(b3, -n3);
  }
}

static cplx corr_t1_eq_t3(int mu, int n2, int n3, int b13, int b2, centre_mp c) {
  (void)n3;
  switch (mu) {
    case 0: return XI * XX(b13, n2 - 6) * G(b2, -(n2 + 2));
    case 1: return conj(XI) * XX(b13, n2 - 2) * G(b2, -(n2 + 2));
    case 2: return XI * XA(b13, n2 - 2) * G(b2, -(n2 + 2));
    case 3: return XI * XX(b13, n2 - 6) * conj(G(b2, n2 - 2));
    case 4: return XI * XA(b13, n2 - 2) * G(b2, -(n2 + 2));
    case 5: return conj(XI) * XA(b13, n2 + 2) * G(b2, -(n2 + 2));
    case 6: return conj(XI) * XX(b13, n2 - 2) * conj(G(b2, n2 - 2));
    case 7: return conj(XI) * XA(b13, n2 + 2) * G(b2, -(n2 + 2));
    default: return WI * WW(b13, n2) * W(b2, -n2);
  }
}

static cplx corr_t2_eq_t3(int mu, int n2, int n3, int b23, int b1, centre_mp c) {
  const int s = n2 + n3;
  switch (mu) {
    case 0: return XI * XX(b23, -(s + 5)) * G(b1, s - 3);
    case 1: return conj(XI) * XX(b23, -(s + 3)) * G(b1, s - 1);
    case 2: return XI * XX(b23, -(s + 5)) * conj(G(b1, -(s + 1)));
    case 3: return XI * XA(b23, -(s + 1)) * G(b1, s - 3);
    case 4: return XI * XA(b23, -(s + 1)) * G(b1, s - 3);
    case 5: return conj(XI) * XX(b23, -(s + 3)) * conj(G(b1, -(s + 3)));
    case 6: return conj(XI) * XA(b23, -(s - 1)) * G(b1, s - 1);
    case 7: return conj(XI) * XA(b23, -(s - 1)) * G(b1, s - 1);
    default: return WI * WW(b23, -s) * W(b1, s);
  }
}

/* Triple-counting term (last column of Table tab:4PCFMCCorr). */
static cplx corr_triple(int mu, int b, centre_mp c) {
  switch (mu) {
    case 0: return XI * XXX_M8(b);
    case 1: return conj(XI) * XXX_M4(b);
    case 2:
    case 3:
    case 4: return XI * XXC_M4(b);
    case 5:
    case 6:
    case 7: return conj(XI) * XXC_0(b);
    default: return WI * WWW_0(b);
  }
}

static size_t ups_index(int mu, int n2, int n3, int b1, int b2, int b3, int N, int nb) {
  const size_t nn = (size_t)(2 * N + 1);
  return (((((size_t)mu * nn + (size_t)(n2 + N)) * nn + (size_t)(n3 + N)) * nb + b1) * nb + b2) *
             nb + b3;
}

int o4_measure(int64_t n_gal, const double* pos, const double* shear, const double* w,
               const double* edges, int nb, int nmax, const uint8_t* centre_mask,
               int corrections, int n_threads, double* ups, double* xi_acc) {
  if (n_gal < 0 || nmax < 0 || check_edges(edges, nb)) return -1;
  if (n_gal == 0) return 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  const int N = nmax;
  double* e2 = (double*)malloc((size_t)(nb + 1) * sizeof(double));
  for (int b = 0; b <= nb; ++b) e2[b] = edges[b] * edges[b];
  cell_list cl;
  if (cell_list_build(&cl, n_gal, pos, edges[nb])) return -2;

  /* the list of centres */
  int64_t n_cen = 0;
  int64_t* cen = (int64_t*)malloc((size_t)n_gal * sizeof(int64_t));
  for (int64_t i = 0; i < n_gal; ++i)
    if (!centre_mask || centre_mask[i]) cen[n_cen++] = i;

  mp_dims d = make_dims(N, nb);
  const int64_t BLOCK = 128;
  cplx* mp = (cplx*)malloc((size_t)BLOCK * d.per_centre * sizeof(cplx));
  const int nn = 2 * N + 1;
  cplx* U = (cplx*)ups;

  for (int64_t c0 = 0; c0 < n_cen; c0 += BLOCK) {
    const int64_t nc = (n_cen - c0 < BLOCK) ? n_cen - c0 : BLOCK;
    /* step A: the centres' multipoles */
#pragma omp parallel for schedule(dynamic)
    for (int64_t t = 0; t < nc; ++t) {
      centre_mp cm = {&d, mp + (size_t)t * d.per_centre};
      centre_multipoles(cen[c0 + t], n_gal, pos, shear, w, e2, &cl, cm);
    }
    /* step B: Upsilon_n and N_n summed over the block's centres, minus the
     * multiple-counting terms.  Each (mu, n2) slab is owned by one thread. */
#pragma omp parallel for schedule(dynamic)
    for (int task = 0; task < NCOMP * nn; ++task) {
      const int mu = task / nn, n2 = task % nn - N;
      for (int n3 = -N; n3 <= N; ++n3)
        for (int b1 = 0; b1 < nb; ++b1)
          for (int b2 = 0; b2 < nb; ++b2)
            for (int b3 = 0; b3 < nb; ++b3) {
              cplx acc = 0.0;
              for (int64_t t = 0; t < nc; ++t) {
                centre_mp c = {&d, mp + (size_t)t * d.per_centre};
                cplx v = upsilon_term(mu, n2, n3, b1, b2, b3, c);
                if (corrections) {
                  if (b1 == b2) v -= corr_t1_eq_t2(mu, n2, n3, b1, b3, c);
                  if (b1 == b3) v -= corr_t1_eq_t3(mu, n2, n3, b1, b2, c);
                  if (b2 == b3) v -= corr_t2_eq_t3(mu, n2, n3, b2, b1, c);
                  if (b1 == b2 && b1 == b3) v += 2.0 * corr_triple(mu, b1, c);
                }
                acc += v;
              }
              U[ups_index(mu, n2, n3, b1, b2, b3, N, nb)] += acc;
            }
    }
    if (xi_acc) {
      cplx* X = (cplx*)xi_acc;
      for (int64_t t = 0; t < nc; ++t) {
        centre_mp c = {&d, mp + (size_t)t * d.per_centre};
        for (int b = 0; b < nb; ++b) {
          X[3 * b + 0] += conj(XI) * G(b, 0);
          X[3 * b + 1] += XI * G(b, -4);
          X[3 * b + 2] += WI * W(b, 0);
        }
      }
    }
  }
  free(mp);
  free(cen);
  free(e2);
  cell_list_free(&cl);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Brute force of the definition.  For centre i and neighbours j, k, l (in radial bins     */
/* Theta1, Theta2, Theta3) the quadruplet contributes                                      */
/*   prod_a w_a gamma^(beta_a)(X_a; zeta_a)  e^{-i n2 phi_ijk} e^{-i n3 phi_ijl}           */
/* with gamma(X; zeta) = -gamma_c e^{-2 i zeta} (Eq. gammatx_def), zeta from Eq. xprojection */
/* (phi_1 = phi_ij, phi_2 = phi_ik, phi_3 = phi_il), beta_a the conjugation pattern of    */
/* Eqs. Gamma0_def..Gamma7_def, and phi_ijk = phi_ik - phi_ij.  N_n uses the weights only. */
/* ------------------------------------------------------------------------------------ */
static const int BETA[8][4] = {{0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0},
                               {0, 0, 0, 1}, {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1}};

static cplx projected(cplx gc, double zeta, int conjugate) {
  return conjugate ? -conj(gc) * cexp(2.0 * I * zeta) : -gc * cexp(-2.0 * I * zeta);
}

int o4_bruteforce(int64_t n_gal, const double* pos, const double* shear, const double* w,
                  const double* edges, int nb, int nmax, const uint8_t* centre_mask,
                  int distinct, double* ups) {
  if (n_gal < 0 || nmax < 0 || check_edges(edges, nb)) return -1;
  const int N = nmax, nn = 2 * N + 1;
  double* e2 = (double*)malloc((size_t)(nb + 1) * sizeof(double));
  for (int b = 0; b <= nb; ++b) e2[b] = edges[b] * edges[b];
  cplx* U = (cplx*)ups;
  int64_t* nbr = (int64_t*)malloc((size_t)(n_gal > 0 ? n_gal : 1) * sizeof(int64_t));
  int* nbin = (int*)malloc((size_t)(n_gal > 0 ? n_gal : 1) * sizeof(int));
  double* nphi = (double*)malloc((size_t)(n_gal > 0 ? n_gal : 1) * sizeof(double));
  cplx* e2n = (cplx*)malloc((size_t)nn * sizeof(cplx));
  cplx* e3n = (cplx*)malloc((size_t)nn * sizeof(cplx));
  for (int64_t i = 0; i < n_gal; ++i) {
    if (centre_mask && !centre_mask[i]) continue;
    int64_t m = 0;
    for (int64_t j = 0; j < n_gal; ++j) {
      if (j == i) continue;
      double dx = pos[2 * j] - pos[2 * i], dy = pos[2 * j + 1] - pos[2 * i + 1];
      int b = radial_bin(dx * dx + dy * dy, e2, nb);
      if (b < 0) continue;
      nbr[m] = j;
      nbin[m] = b;
      nphi[m] = atan2(dy, dx);
      ++m;
    }
    const cplx gi = shear[2 * i] + I * shear[2 * i + 1];
    for (int64_t p = 0; p < m; ++p)
      for (int64_t q = 0; q < m; ++q)
        for (int64_t r = 0; r < m; ++r) {
          const int64_t j = nbr[p], k = nbr[q], l = nbr[r];
          if (distinct && (j == k || j == l || k == l)) continue;
          const double p1 = nphi[p], p2 = nphi[q], p3 = nphi[r];
          const double zeta[4] = {0.5 * (p1 + p3), p1, p2, p3};
          const int64_t idx[4] = {i, j, k, l};
          const cplx gc[4] = {gi, shear[2 * j] + I * shear[2 * j + 1],
                              shear[2 * k] + I * shear[2 * k + 1],
                              shear[2 * l] + I * shear[2 * l + 1]};
          double wprod = 1.0;
          for (int a = 0; a < 4; ++a) wprod *= w[idx[a]];
          cplx val[NCOMP];
          for (int mu = 0; mu < 8; ++mu) {
            cplx v = wprod;
            for (int a = 0; a < 4; ++a) v *= projected(gc[a], zeta[a], BETA[mu][a]);
            val[mu] = v;
          }
          val[8] = wprod;
          for (int t = 0; t < nn; ++t) {
            e2n[t] = cexp(-I * (double)(t - N) * (p2 - p1));
            e3n[t] = cexp(-I * (double)(t - N) * (p3 - p1));
          }
          for (int mu = 0; mu < NCOMP; ++mu)
            for (int a2 = 0; a2 < nn; ++a2)
              for (int a3 = 0; a3 < nn; ++a3)
                U[ups_index(mu, a2 - N, a3 - N, nbin[p], nbin[q], nbin[r], N, nb)] +=
                    val[mu] * e2n[a2] * e3n[a3];
        }
  }
  free(nbr);
  free(nbin);
  free(nphi);
  free(e2n);
  free(e3n);
  free(e2);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Multipoles -> real space.  Eq. Multipole2RealConversion gives the angular density     */
/*   Upsilon(phi12, phi13) = (2 pi)^-2 sum_n Upsilon_n e^{i n2 phi12} e^{i n3 phi13};      */
/* integrating it over the angular bin [Phi_lo, Phi_hi) of each axis gives the quadruplet */
/* sums of Eq. QuadrupletUpsilon / Eq. TripletNorm for that bin, and their ratio is the    */
/* estimator of Eq. 4PCF_quadrupletestimator.                                              */
/* ------------------------------------------------------------------------------------ */
static cplx bin_integral(int n, double lo, double hi) {
  if (n == 0) return hi - lo;
  return (cexp(I * (double)n * hi) - cexp(I * (double)n * lo)) / (I * (double)n);
}

int o4_to_real_space(const double* ups, int nb, int nmax, int nphi, double* gamma,
                     double* norm) {
  if (nb < 1 || nmax < 0 || nphi < 1) return -1;
  const int N = nmax, nn = 2 * N + 1;
  const double two_pi = 2.0 * M_PI;
  cplx* E = (cplx*)malloc((size_t)nn * nphi * sizeof(cplx));
  for (int t = 0; t < nn; ++t)
    for (int p = 0; p < nphi; ++p)
      E[(size_t)t * nphi + p] = bin_integral(t - N, two_pi * p / nphi, two_pi * (p + 1) / nphi);
  const cplx* U = (const cplx*)ups;
  cplx* Gm = (cplx*)gamma;
  const size_t nb3 = (size_t)nb * nb * nb, nph2 = (size_t)nphi * nphi;
#pragma omp parallel for schedule(dynamic)
  for (int64_t tri = 0; tri < (int64_t)nb3; ++tri) {
    const int b1 = (int)(tri / ((int64_t)nb * nb)), b2 = (int)((tri / nb) % nb),
              b3 = (int)(tri % nb);
    double* nrm = (double*)malloc(nph2 * sizeof(double));
    for (int mu = 8; mu >= 0; --mu) {
      for (int p = 0; p < nphi; ++p)
        for (int q = 0; q < nphi; ++q) {
          cplx acc = 0.0;
          for (int a2 = 0; a2 < nn; ++a2)
            for (int a3 = 0; a3 < nn; ++a3)
              acc += U[ups_index(mu, a2 - N, a3 - N, b1, b2, b3, N, nb)] *
                     E[(size_t)a2 * nphi + p] * E[(size_t)a3 * nphi + q];
          acc /= two_pi * two_pi;
          const size_t o = (size_t)p * nphi + q;
          if (mu == 8) {
            nrm[o] = creal(acc);
            norm[(size_t)tri * nph2 + o] += creal(acc);
          } else {
            cplx g = (nrm[o] != 0.0) ? acc / nrm[o] : 0.0;
            Gm[((size_t)mu * nb3 + (size_t)tri) * nph2 + o] += g;
          }
        }
    }
    free(nrm);
  }
  free(E);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Fourth-order aperture measures.                                                        */
/* With Q_theta of Eq. CrittendenQ, Q(|v|) e^{-2i arg v} = v^{*2} e^{-|v|^2/2theta^2} /    */
/* (4 pi theta^4), and e^{+2i arg v} gives v^2 instead.  Inserting Eq. MapGamma four times */
/* for apertures at a common centre X, writing the galaxies as Y_0 = X + y, Y_a = Y_0 +    */
/* vartheta_a, and converting the Cartesian correlator to Gamma^x with Eq. gammatx_def and */
/* Eq. xprojection gives                                                                   */
/*  <M_beta> = int d^2vt1 d^2vt2 d^2vt3 Gamma_mu e^{2i sum_a s_a zeta_a} (4 pi theta^4)^-4 */
/*             exp(-sum_a |d_a|^2 / 2 theta^2) J_beta,                                      */
/*  J_beta  = int d^2z prod_{beta_a=0} (z + d_a)^{*2} prod_{beta_a=1} (z + d_a)^2           */
/*            exp(-2 |z|^2 / theta^2),  d_a = vartheta_a - (sum_b vartheta_b)/4,            */
/* s_a = +1 (-1) for an unconjugated (conjugated) aperture, vartheta_0 = 0.  Only equal    */
/* powers of z and z^* survive the z integral: int |z|^{2p} e^{-2|z|^2/theta^2} d^2z =     */
/* pi p! (theta^2/2)^{p+1}.  The integrand is invariant under a common rotation, so       */
/* phi_1 = 0 and the phi_1 integral gives 2 pi; d^2vt = vt dvt dphi.                       */
/* ------------------------------------------------------------------------------------ */
static void poly_mul_lin2(cplx* poly, int* deg, cplx root) {
  /* multiply poly (coefficients of t^0..t^deg) by (t + root)^2 */
  for (int rep = 0; rep < 2; ++rep) {
    cplx nxt[16] = {0};
    for (int p = 0; p <= *deg; ++p) {
      nxt[p + 1] += poly[p];
      nxt[p] += poly[p] * root;
    }
    *deg += 1;
    for (int p = 0; p <= *deg; ++p) poly[p] = nxt[p];
  }
}

void o4_map4_filter(int mu, double theta, double t1, double t2, double t3, double phi12,
                    double phi13, double* out) {
  const cplx vt[4] = {0.0, t1, t2 * cexp(I * phi12), t3 * cexp(I * phi13)};
  const cplx cen = (vt[1] + vt[2] + vt[3]) / 4.0;
  cplx d[4];
  double sumd2 = 0.0;
  for (int a = 0; a < 4; ++a) {
    d[a] = vt[a] - cen;
    sumd2 += creal(d[a] * conj(d[a]));
  }
  cplx P[16] = {1.0}, R[16] = {1.0};
  int dP = 0, dR = 0;
  for (int a = 0; a < 4; ++a) {
    if (BETA[mu][a]) poly_mul_lin2(R, &dR, d[a]);  /* (z + d_a)^2, powers of z */
    else poly_mul_lin2(P, &dP, conj(d[a]));        /* (z^* + d_a^*)^2, powers of z^* */
  }
  const double h = 0.5 * theta * theta;
  cplx J = 0.0;
  double fact = 1.0;
  for (int p = 0; p <= dP && p <= dR; ++p) {
    if (p > 0) fact *= (double)p;
    J += P[p] * R[p] * M_PI * fact * pow(h, (double)(p + 1));
  }
  /* 2 sum_a s_a zeta_a with zeta_0 = (phi1+phi3)/2, zeta_1 = phi1 = 0, zeta_2 = phi12,
   * zeta_3 = phi13 */
  const double zeta[4] = {0.5 * phi13, 0.0, phi12, phi13};
  double ph = 0.0;
  for (int a = 0; a < 4; ++a) ph += 2.0 * (BETA[mu][a] ? -1.0 : 1.0) * zeta[a];
  const double q0 = 4.0 * M_PI * theta * theta * theta * theta;
  cplx F = 2.0 * M_PI * t1 * t2 * t3 * cexp(I * ph) * J * exp(-sumd2 / (2.0 * theta * theta)) /
           (q0 * q0 * q0 * q0);
  out[0] = creal(F);
  out[1] = cimag(F);
}

/* E/B split: with M_a = P_a + i X_a (P = M_ap, X = M_perp), every conjugation pattern
 * beta of <M_0 M_1 M_2 M_3> is sum_b prod_a c(beta_a, b_a) <b_0 b_1 b_2 b_3>; the 8
 * patterns of Eq. M4Ordering and their complements (complex conjugates) give all 16, and
 * P = (M + M^*)/2, X = (M - M^*)/(2i) invert it. */
static int pattern_code(const int* beta) { return beta[0] * 8 + beta[1] * 4 + beta[2] * 2 + beta[3]; }

/* component order of Eq. 4PCF_rawcomponents, t -> 0 (M_ap), x -> 1 (M_perp); the
 * repeated "xxtx" of the printed list is read as "xxxt" (the only missing combination) */
static const char* EB_ORDER[16] = {"tttt", "xttt", "txtt", "ttxt", "tttx", "ttxx",
                                   "txtx", "txxt", "xttx", "xtxt", "xxtt", "txxx",
                                   "xtxx", "xxtx", "xxxt", "xxxx"};

static void eb_from_patterns(const cplx* D /* [16] by pattern code */, double* out16) {
  for (int c = 0; c < 16; ++c) {
    cplx acc = 0.0;
    for (int code = 0; code < 16; ++code) {
      int beta[4] = {(code >> 3) & 1, (code >> 2) & 1, (code >> 1) & 1, code & 1};
      cplx coef = 1.0;
      for (int a = 0; a < 4; ++a) {
        if (EB_ORDER[c][a] == 't') coef *= 0.5;
        else coef *= beta[a] ? 0.5 * I : -0.5 * I;
      }
      acc += coef * D[code];
    }
    out16[c] += creal(acc);
  }
}

static void patterns_from_m4(const cplx* m4, cplx* D) {
  for (int mu = 0; mu < 8; ++mu) {
    int comp[4];
    for (int a = 0; a < 4; ++a) comp[a] = 1 - BETA[mu][a];
    D[pattern_code(BETA[mu])] = m4[mu];
    D[pattern_code(comp)] = conj(m4[mu]);
  }
}

void o4_eb_from_m4(const double* m4, double* out16) {
  cplx D[16];
  patterns_from_m4((const cplx*)m4, D);
  eb_from_patterns(D, out16);
}

int o4_map4(const double* ups, const double* edges, int nb, int nmax, int nphi,
            const double* ap_radii, int n_ap, const double* xi_pm, double* m4, double* map4,
            double* disc) {
  if (check_edges(edges, nb) || nmax < 0 || nphi < 1 || n_ap < 0) return -1;
  const size_t nb3 = (size_t)nb * nb * nb, nph2 = (size_t)nphi * nphi;
  double* gam = (double*)calloc(8 * nb3 * nph2 * 2, sizeof(double));
  double* nrm = (double*)calloc(nb3 * nph2, sizeof(double));
  if (!gam || !nrm) return -2;
  o4_to_real_space(ups, nb, nmax, nphi, gam, nrm);
  const cplx* Gm = (const cplx*)gam;
  /* radial bins: area element A_b = int vt dvt, representative radius = vt-weighted mean */
  double* A = (double*)malloc((size_t)nb * sizeof(double));
  double* tb = (double*)malloc((size_t)nb * sizeof(double));
  for (int b = 0; b < nb; ++b) {
    const double lo = edges[b], hi = edges[b + 1];
    A[b] = 0.5 * (hi * hi - lo * lo);
    tb[b] = (2.0 / 3.0) * (hi * hi * hi - lo * lo * lo) / (hi * hi - lo * lo);
  }
  const double dphi = 2.0 * M_PI / nphi;
  cplx* M = (cplx*)m4;
  for (int ia = 0; ia < n_ap; ++ia) {
    const double th = ap_radii[ia];
    cplx acc[8] = {0};
#pragma omp parallel for schedule(dynamic)
    for (int64_t tri = 0; tri < (int64_t)nb3; ++tri) {
      const int b1 = (int)(tri / ((int64_t)nb * nb)), b2 = (int)((tri / nb) % nb),
                b3 = (int)(tri % nb);
      const double vol = A[b1] / tb[b1] * A[b2] / tb[b2] * A[b3] / tb[b3] * dphi * dphi;
      cplx loc[8] = {0};
      for (int p = 0; p < nphi; ++p)
        for (int q = 0; q < nphi; ++q)
          for (int mu = 0; mu < 8; ++mu) {
            double F[2];
            o4_map4_filter(mu, th, tb[b1], tb[b2], tb[b3], (p + 0.5) * dphi, (q + 0.5) * dphi, F);
            loc[mu] += Gm[((size_t)mu * nb3 + (size_t)tri) * nph2 + (size_t)p * nphi + q] *
                       (F[0] + I * F[1]) * vol;
          }
#pragma omp critical
      for (int mu = 0; mu < 8; ++mu) acc[mu] += loc[mu];
    }
    for (int mu = 0; mu < 8; ++mu) M[(size_t)ia * 8 + mu] += acc[mu];
    o4_eb_from_m4((const double*)acc, map4 + (size_t)ia * 16);
    /* Gaussian (disconnected) part: <M M^*> and <M M> of one aperture from xi_+ and
     * xi_- with T_+(x) = (x^4 - 16 x^2 + 32)/128 e^{-x^2/4}, T_-(x) = x^4/128 e^{-x^2/4},
     * obtained with the same Gaussian z-integral for two apertures; Wick's theorem
     * pairs them into every conjugation pattern of four apertures. */
    if (xi_pm) {
      cplx Am = 0.0;
      double Bp = 0.0;
      for (int b = 0; b < nb; ++b) {
        const double x = tb[b] / th, g = exp(-0.25 * x * x);
        const double Tp = (x * x * x * x - 16.0 * x * x + 32.0) / 128.0 * g;
        const double Tm = x * x * x * x / 128.0 * g;
        Bp += xi_pm[4 * b + 0] * Tp * A[b] / (th * th);
        Am += (xi_pm[4 * b + 2] + I * xi_pm[4 * b + 3]) * Tm * A[b] / (th * th);
      }
      cplx D[16];
      for (int code = 0; code < 16; ++code) {
        int be[4] = {(code >> 3) & 1, (code >> 2) & 1, (code >> 1) & 1, code & 1};
        cplx pair[4][4];
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            pair[a][b] = (be[a] == be[b]) ? (be[a] ? conj(Am) : Am) : (cplx)Bp;
        D[code] = pair[0][1] * pair[2][3] + pair[0][2] * pair[1][3] + pair[0][3] * pair[1][2];
      }
      eb_from_patterns(D, disc + (size_t)ia * 16);
    }
  }
  free(A);
  free(tb);
  free(gam);
  free(nrm);
  return 0;
}
