/*
 * oracle4pcf.h -- plain FP64 CPU oracle for the multipole estimator of the shear
 * four-point correlation function (Porth, Silvestre-Rosello, Schneider, Larma 2025,
 * "Towards an application of fourth-order shear statistics II", arXiv:2509.07974).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; the product
 * never links, loads or calls it.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may use it.  It shares no code, header,
 * table or constant with the GPU library.
 *
 * Array layouts (all row-major, complex values stored as interleaved re,im doubles):
 *   pos     [n_gal][2]   flat-sky x, y
 *   shear   [n_gal][2]   Cartesian gamma_1, gamma_2 (gamma_c = g1 + i g2)
 *   w       [n_gal]      weights
 *   edges   [nb+1]       radial bin edges, strictly increasing, edges[0] > 0
 *   ups     [9][2N+1][2N+1][nb][nb][nb][2]  mu = 0..7 natural components, mu = 8 the
 *                                            normalisation; index n2+N, n3+N.
 * All functions ACCUMULATE into their outputs (callers zero them).
 * Return 0 on success, negative on invalid arguments.
 */
#ifndef ORACLE4PCF_H
#define ORACLE4PCF_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Factorised multipole estimator: per-centre G_n / W_n (Eq. 4PCFUpsilon0 and the seven
 * equations after it, Eq. Nnmultipoles), summed over centres, then (if corrections != 0)
 * the multiple-counting terms of Table tab:4PCFMCCorr (App. A.1) removed.
 * centre_mask may be NULL (every galaxy is a centre).  xi_acc, if not NULL, receives
 * [nb][6] = (sum x_i^* G_0, sum x_i G_-4, sum w_i W_0) per radial bin (complex each). */
int o4_measure(int64_t n_gal, const double* pos, const double* shear, const double* w,
               const double* edges, int nb, int nmax, const uint8_t* centre_mask,
               int corrections, int n_threads, double* ups, double* xi_acc);

/* Brute force of the definition (Eq. QuadrupletUpsilon, Eq. TripletNorm projected on the
 * multipole basis as in Eq. 4PCFUpsilon0_Derivation), over ordered quadruplets of
 * pairwise-distinct galaxy indices (or all index combinations if distinct == 0).  O(N^4):
 * tiny catalogues only. */
int o4_bruteforce(int64_t n_gal, const double* pos, const double* shear, const double* w,
                  const double* edges, int nb, int nmax, const uint8_t* centre_mask,
                  int distinct, double* ups);

/* Multipoles -> real space (Eq. Multipole2RealConversion), bin-integrated over nphi
 * uniform angular bins on [0, 2 pi).  norm [nb]^3[nphi][nphi] = quadruplet weight per
 * bin; gamma [8][nb]^3[nphi][nphi][2] = Upsilon / norm (0 where norm == 0). */
int o4_to_real_space(const double* ups, int nb, int nmax, int nphi, double* gamma,
                     double* norm);

/* Integrand kernel of Eq. 4PCF2M4 for the Crittenden filter (Eq. CrittendenQ), derived in
 * closed form (aperture centre integrated analytically).  Returns F_mu, including the
 * Jacobian 2 pi t1 t2 t3, into out[2]. */
void o4_map4_filter(int mu, double theta, double t1, double t2, double t3, double phi12,
                    double phi13, double* out);

/* Fourth-order aperture statistics from the multipoles: m4 [n_ap][8][2] (Eq. M4Ordering),
 * map4 [n_ap][16] E/B components ordered as Eq. 4PCF_rawcomponents, disc [n_ap][16] the
 * Gaussian part built from xi_pm ([nb][4] = xi+ re,im, xi- re,im; may be NULL -> zero). */
int o4_map4(const double* ups, const double* edges, int nb, int nmax, int nphi,
            const double* ap_radii, int n_ap, const double* xi_pm, double* m4, double* map4,
            double* disc);

/* E/B decomposition of Eq. M4Ordering correlators (8 complex) into 16 real moments. */
void o4_eb_from_m4(const double* m4, double* out16);

#ifdef __cplusplus
}
#endif
#endif
