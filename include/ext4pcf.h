/*
 * ext4pcf.h -- C ABI of the GB300 (sm_103a) implementation of the quadratic-scaling
 * multipole estimator of the shear four-point correlation function of Porth,
 * Silvestre-Rosello, Schneider & Larma, arXiv:2509.07974 ("the paper").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Positions are flat-sky (x, y) in any angular unit; radial bin edges use the same unit.
 *  - Shears are Cartesian (gamma_1, gamma_2), gamma_c = gamma_1 + i gamma_2 (paper Sect. 2.1).
 *  - Complex values are interleaved (re, im) doubles.
 *  - Multipole output ("upsilon") layout, row-major:
 *        [n_cat][9][2N+1][2N+1][nb][nb][nb][2]
 *    index 0..7 along the second axis are the natural components Upsilon_mu of the
 *    x-projection (paper Eq. 4PCFUpsilon0 and the seven equations after it), index 8 is
 *    the normalisation N_n (Eq. Nnmultipoles); the next two axes are n2+N and n3+N
 *    (N = n_max); the three bin axes are Theta1, Theta2, Theta3.  Every ordered bin triple
 *    is stored.
 *  - Outputs are ACCUMULATED INTO: the caller zeroes them before the first call; results of
 *    several calls (patches, checkpointed chunks of a catalogue) add up.
 *  - Ownership: the caller owns every input and output buffer; the context owns its
 *    scratch memory (grown on demand, released by ext4pcf_destroy).
 *  - Pointers documented as "device or host" may point to either; host buffers are copied
 *    to the device inside the call (and host outputs copied back), which makes the call
 *    synchronous.  ext4pcf_measure and ext4pcf_measure3 with device pointers (and no
 *    `stats`) are stream-ordered on the configured stream and return after enqueueing: the
 *    cell grid is chosen on the device and no value is read back.  A bounded device-side wait
 *    that ran out, or positions that are not all finite, are recorded in the context's status
 *    word and reported (EXT4PCF_E_TIMEOUT, EXT4PCF_E_INVALID_ARG) by the next call that
 *    synchronises: ext4pcf_synchronize, or ext4pcf_measure with `stats` or host outputs.
 *    Scratch buffers grow on the first call of a size, and tensor-core work tables are
 *    uploaded on the first call of an (n_bins, n_max): both synchronise, so make one such
 *    call before capturing the stream into a CUDA graph.
 *  - Errors: every entry point returns EXT4PCF_OK (0) or a negative code; no exception
 *    crosses the ABI.  ext4pcf_last_error() gives a message for the last failure.  A
 *    context may be used by one host thread at a time.
 */
#ifndef EXT4PCF_H
#define EXT4PCF_H

#include <stdint.h>

#if defined(__GNUC__)
#define EXT4PCF_API __attribute__((visibility("default")))
#else
#define EXT4PCF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ext4pcf_ctx ext4pcf_ctx;

enum {
  EXT4PCF_OK = 0,
  EXT4PCF_E_INVALID_ARG = -1, /* bad sizes, unsorted or non-positive bins, n_max < 0 ... */
  EXT4PCF_E_OOM = -2,         /* device allocation failed */
  EXT4PCF_E_CUDA = -3,        /* a CUDA runtime call failed */
  EXT4PCF_E_TIMEOUT = -4,     /* a bounded device-side wait gave up (status word set) */
  EXT4PCF_E_UNSUPPORTED = -5  /* no sm_103 device, or a size beyond a kernel's limits */
};

/* Arithmetic of ext4pcf_measure. */
typedef enum {
  EXT4PCF_FP64 = 0,      /* FP64 gather, FP64 contraction and corrections (CUDA cores) */
  EXT4PCF_FP32 = 1,      /* FP32 gather and contraction, FP64 accumulation across waves */
  EXT4PCF_TF32 = 2,      /* FP32 gather, tensor-core contraction (tcgen05 kind::tf32) */
  EXT4PCF_3XTF32 = 3,    /* as TF32 with hi/lo split operands, three passes */
  EXT4PCF_SPLIT_BF16 = 4,/* tensor-core contraction (kind::f16, bf16 hi/lo, three passes) */
  EXT4PCF_SPLIT_F16 = 5  /* kind::f16 with fp16 hi/lo (22 bits per operand, as 3XTF32), three
                            passes at twice the tf32 rate; every row of the wave's multipoles
                            is scaled by a power of two so that its largest component over the
                            wave lies in [2^6, 2^7) (products stay below 2^15, inside the fp16
                            range), and the scales are undone exactly in FP64 */
} ext4pcf_precision;

typedef struct {
  int device;              /* CUDA device ordinal */
  void* stream;            /* cudaStream_t to enqueue on (NULL = legacy default stream) */
  int precision;           /* ext4pcf_precision */
  int autotune;            /* 1: the first measure call of an (precision, n_max, n_bins) times its
                              first waves at 2048, 4096, 8192 and 16384 centres and keeps the
                              fastest per centre for the context (those waves synchronise; needs
                              no centre mask and enough centres, else the default is kept) */
  int64_t workspace_bytes; /* cap on the per-wave scratch of ext4pcf_measure (records, staging):
                              the wave shrinks by halves to fit; 0 = no cap */
  int64_t timeout_cycles;  /* bound on every device-side wait (0 = default) */
  int deterministic;       /* 1: fixed summation order (always honoured at present) */
  int wave_centres;        /* centres per contraction wave (0 = autotuned or 8192, 4096 for FP64) */
  /* Tree approximation of the neighbour multipoles (paper Sect. 3.2, App. F.3, Eq.
   * NPCF_treeestimator): radial bins far from the centre take their neighbours from reduced
   * catalogues, the galaxies of each cell of side Delta_d = tree_delta1 2^(d-1) (d = 1 ..
   * tree_levels, grids anchored at each catalogue's lower bounding-box corner) replaced by one
   * galaxy at their weighted centre of mass with the summed w and w gamma.  A bin uses the
   * coarsest level with Theta_lo / Delta_d >= tree_rmin, the galaxies when none qualifies.  The
   * centres stay the galaxies.  tree_delta1 = 0 (or tree_levels = 0): exact multipoles.  With
   * the tree in use a measure call reads the reduced catalogues' sizes back (one
   * synchronisation). */
  double tree_delta1;
  int tree_levels;         /* 0 .. 8 */
  double tree_rmin;
} ext4pcf_config;

typedef struct {
  int64_t pairs;   /* (centre, neighbour) pairs with separation inside the radial bins */
  int64_t centres; /* galaxies that acted as centres */
  int64_t waves;   /* contraction waves launched */
  int64_t launches; /* kernels launched by the call */
  double ms_grid, ms_gather, ms_contract, ms_correct, ms_total; /* CUDA-event times */
  int64_t wave_centres; /* wave size of the call after any autotuning (at most its largest wave) */
} ext4pcf_stats;

/* Create a context on cfg->device.  Fails with EXT4PCF_E_UNSUPPORTED unless the device is
 * compute capability 10.3 (GB300).  *out receives the handle. */
EXT4PCF_API int ext4pcf_create(ext4pcf_ctx** out, const ext4pcf_config* cfg);

/* Release the context and all its scratch memory (synchronises its stream). */
EXT4PCF_API int ext4pcf_destroy(ext4pcf_ctx* ctx);

/* Wait for the work enqueued on the context's stream and report what its status word
 * recorded since it was last read (then clear it): EXT4PCF_OK, EXT4PCF_E_TIMEOUT (a bounded
 * device-side wait in the tensor-core contraction ran out; that call's results are not
 * valid), EXT4PCF_E_INVALID_ARG (positions that were not all finite), or EXT4PCF_E_CUDA. */
EXT4PCF_API int ext4pcf_synchronize(ext4pcf_ctx* ctx);

/* Multipoles of the shear 4PCF (paper Sect. 3.1 and App. A.1).
 * For every centre galaxy i and radial bin Theta, the neighbour multipoles
 *   G_n(theta_i, Theta) = sum_j w_j gamma_c,j e^{i n phi_ij}, W_n likewise with w_j
 * (phi_ij the polar angle of theta_j - theta_i, bin membership Theta_lo^2 <= r^2 <
 * Theta_hi^2) are accumulated, contracted into Upsilon_{mu,n}(Theta1,Theta2,Theta3) and
 * N_n (Eq. 4PCFUpsilon0 ff., Eq. Nnmultipoles) and the double- and triple-counting terms
 * of Table tab:4PCFMCCorr are removed, so that only quadruplets of distinct galaxy indices
 * remain.
 *   positions   device or host, double [n_gal][2]
 *   shears      device or host, double [n_gal][2]
 *   weights     device or host, double [n_gal]
 *   n_gal       total galaxies over all catalogues (>= 0)
 *   radial_bins host, double [n_bins+1], strictly increasing, radial_bins[0] > 0
 *   n_bins      1..32 (1..16 for the tensor-core precisions TF32, 3XTF32, SPLIT_BF16 and SPLIT_F16, whose
 *               B tile holds at most 64 columns, 4 per bin; larger n_bins return
 *               EXT4PCF_E_UNSUPPORTED before any work);  n_max >= 0 (<= 40).  A centre's
 *               record, n_bins (14 n_max + 18) complex values, must also fit the gather's
 *               shared memory: every n_max up to n_bins = 16; at n_bins = 20, 24, 28, 32,
 *               n_max <= 37, 31, 26, 23 (FP32 gather, every precision but FP64) or
 *               n_max <= 40, 37, 31, 27 (FP64).  Larger records return
 *               EXT4PCF_E_UNSUPPORTED when the first wave is gathered.
 *   cat_offsets host, int64 [n_cat+1] or NULL: catalogue k is galaxies
 *               [cat_offsets[k], cat_offsets[k+1]); NULL means one catalogue (n_cat = 1)
 *   centre_mask device or host, uint8 [n_gal] or NULL: only galaxies with a non-zero entry
 *               act as centres (all galaxies act as neighbours)
 *   upsilon     device or host, double, layout above, accumulated into
 *   xi_acc      device or host, double [n_cat][n_bins][3][2] or NULL: accumulates
 *               (sum_i x_i^* G_0, sum_i x_i G_-4, sum_i w_i W_0) per bin, x_i = w_i gamma_c,i
 *               (xi_+ and xi_- are the first two over the third)
 *   stats       host or NULL */
EXT4PCF_API int ext4pcf_measure(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                    const double* weights, int64_t n_gal, const double* radial_bins,
                    int n_bins, int n_max, const int64_t* cat_offsets, int n_cat,
                    const uint8_t* centre_mask, double* upsilon, double* xi_acc,
                    ext4pcf_stats* stats);

/* Batched form of ext4pcf_measure: many catalogues (mocks, or the overlapping patches of one
 * survey) in one call, each catalogue's result added into an output slot.
 *   out_slot    host, int [n_cat] or NULL: catalogue k accumulates into slot out_slot[k]
 *               (0 <= out_slot[k] < n_out); NULL means slot k (n_out = n_cat, as
 *               ext4pcf_measure).  Patches of one survey share slot 0: with a centre mask
 *               marking each patch's core, every galaxy is a centre exactly once and its
 *               neighbours come from the patch's core and margin.
 *   upsilon     [n_out][...] and xi_acc [n_out][n_bins][3][2], otherwise as ext4pcf_measure.
 * The grids of all catalogues are built first, then the centres are processed in waves.  In
 * the SPLIT_F16 form a wave packs the centres of several catalogues (runs starting at
 * multiples of 64 records) whenever their numbers are known on the host (no mask, or a host
 * mask), so that every kernel launch covers many small catalogues; the other forms, and
 * catalogues with a device-resident mask, take one catalogue per wave.  Every output is
 * written by one thread block per kernel in a fixed order (no atomics): results are bitwise
 * reproducible for a given configuration and wave size. */
EXT4PCF_API int ext4pcf_measure_batch(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                    const double* weights, int64_t n_gal, const double* radial_bins, int n_bins,
                    int n_max, const int64_t* cat_offsets, int n_cat, const int* out_slot,
                    int n_out, const uint8_t* centre_mask, double* upsilon, double* xi_acc,
                    ext4pcf_stats* stats);

/* Per-centre neighbour multipoles (the gather of ext4pcf_measure, its output kept): for each
 * requested galaxy the record of sums over its neighbours j in each radial bin, u = e^{i phi_ij},
 * x = w gamma_c, as complex FP64 pairs (the gather runs in FP64 for EXT4PCF_FP64, in FP32
 * otherwise), with the tree approximation of the configuration if set:
 *   G_n   = sum x u^n          n = -2N-3 .. 2N-1   [(4N+3)][n_bins]
 *   W_m   = sum w u^m          m = 0 .. 2N         [(2N+1)][n_bins]   (W_-m = conj W_m)
 *   XX_n  = sum x^2 u^n        n = -2N-6 .. 2N-2   [(4N+5)][n_bins]
 *   XA_m  = sum |x|^2 u^m      m = 0 .. 2N+2       [(2N+3)][n_bins]
 *   WW_m  = sum w^2 u^m        m = 0 .. 2N         [(2N+1)][n_bins]
 *   TR    = sum x^3 u^-8, x^3 u^-4, x^2 x^* u^-4, x^2 x^*, w^3   [5][n_bins]
 * concatenated in this order, the bin fastest: rec = (14N + 18) n_bins complex values a centre.
 *   centres   host, int64 [n_centres]: indices into the catalogue (0 <= centre < n_gal)
 *   records   device or host, double [n_centres][rec][2]
 * One catalogue; synchronises when records is host memory. */
EXT4PCF_API int ext4pcf_multipoles(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                    const double* weights, int64_t n_gal, const double* radial_bins, int n_bins,
                    int n_max, const int64_t* centres, int64_t n_centres, double* records);

/* Multipoles -> real space (paper Eq. Multipole2RealConversion, FP64).  The angular
 * density is integrated over n_phi uniform bins of [0, 2 pi) on each of phi_12, phi_13,
 * giving per bin the quadruplet sums of Eq. QuadrupletUpsilon / Eq. TripletNorm; their
 * ratio is the estimator of Eq. 4PCF_quadrupletestimator.
 *   upsilon device, one catalogue, layout above
 *   gamma   device, double [8][nb][nb][nb][n_phi][n_phi][2], accumulated: Upsilon / N
 *           (0 where N == 0)
 *   norm    device, double [nb][nb][nb][n_phi][n_phi], accumulated: N per bin */
EXT4PCF_API int ext4pcf_to_real_space(ext4pcf_ctx* ctx, const double* upsilon, int n_bins, int n_max,
                          int n_phi, double* gamma, double* norm);

/* Fourth-order aperture measures for the filter of Eq. CrittendenQ (paper Sect. 5, FP64).
 * The real-space 4PCF is formed on the fly (never stored) and integrated with the
 * closed-form kernel of Eq. 4PCF2M4 (aperture centre integrated analytically) over the
 * radial bins (area element (hi^2 - lo^2)/2 at the r-weighted mean radius) and n_phi
 * angular bins.
 *   upsilon     device, one catalogue
 *   radial_bins host [n_bins+1];  ap_radii host [n_ap]
 *   xi_acc      device or host, [n_bins][3][2] accumulators written by ext4pcf_measure
 *               (xi_+ = first / third, xi_- = second / third per bin), or NULL
 *   m4          host [n_ap][8][2]: the correlators of Eq. M4Ordering (accumulated)
 *   map4_eb     host [n_ap][16]: E/B moments in the order of Eq. 4PCF_rawcomponents
 *   map4_disc   host [n_ap][16] or NULL: Gaussian part built from xi_+- (Wick pairs of
 *               <M M> and <M M^*>, each an integral of xi_+- with the two-point filters
 *               T_+- of the same filter), same order; connected = map4_eb - map4_disc */
EXT4PCF_API int ext4pcf_to_map4(ext4pcf_ctx* ctx, const double* upsilon, const double* radial_bins,
                    int n_bins, int n_max, int n_phi, const double* ap_radii, int n_ap,
                    const double* xi_acc, double* m4, double* map4_eb, double* map4_disc);

/* The real-space transform of ext4pcf_to_real_space for callers that cannot allocate device
 * memory (no cudaMalloc, cudaFree or allocating library routine is called, and no context
 * is needed).  The paper has no counterpart: this is a deployment variant.  Scratch lives
 * in one 16 MiB device array inside the library, held by every GPU that loads it until the
 * process exits, so the sizes must satisfy
 *     n_bins^3 * n_phi^2 * 8 (rounded up to 256) + (2 n_max + 1) * n_phi * 16 <= 16 MiB
 * (for example n_bins = 10 with n_phi <= 45, or n_bins = 8 with n_phi <= 63); larger sizes
 * return EXT4PCF_E_UNSUPPORTED before any work is enqueued.
 *   upsilon, gamma, norm  device pointers with the layouts of ext4pcf_to_real_space;
 *                         gamma and norm are accumulated into
 *   stream                cudaStream_t to enqueue on (NULL = legacy default stream)
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The call is stream-ordered and returns
 * after enqueueing.  All calls share the array: calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Returns EXT4PCF_OK, EXT4PCF_E_INVALID_ARG (null or host pointers, sizes out of range),
 * EXT4PCF_E_UNSUPPORTED (beyond the scratch size) or EXT4PCF_E_CUDA. */
EXT4PCF_API int ext4pcf_to_real_space_noalloc(const double* upsilon, int n_bins, int n_max, int n_phi,
                                              double* gamma, double* norm, void* stream);

/* Direct estimator of <M_ap^2> and <M_ap^4> (paper Sect. 5.2, Eq. MapDirectEstimator) for the
 * filter Q_theta of Eq. CrittendenQ, cut at |vartheta_i - vartheta| < 4 theta.  For each
 * aperture (centre vartheta, radius theta) with a_i = w_i Q_theta,i gamma_t,i (gamma_t the real
 * part of Eq. gammatx_def about the centre), the distinct quadruplet sums over the galaxies
 * inside the cut are 4! e_4(a) (numerator) and 4! e_4(w) (denominator), e_k the elementary
 * symmetric polynomials, computed from the power sums of a and w (Newton's identities):
 * linear in the galaxies.  Per-galaxy terms are FP32; the power sums are kept as FP32 (hi, lo)
 * pairs (error-free two-sum) and combined per aperture in FP64.
 *   positions, shears, weights  device or host, as for ext4pcf_measure (one catalogue)
 *   n_gal           0 .. 2^31-1
 *   thetas          host, double [n_theta], finite and > 0 (1 <= n_theta <= 4096)
 *   centres         device or host, double [n_centres][2]: aperture centres, those of radius
 *                   thetas[t] in rows centre_offsets[t] .. centre_offsets[t+1]-1 (the caller
 *                   chooses them, e.g. a lattice at least 4 theta inside the field)
 *   centre_offsets  host, int64 [n_theta+1], centre_offsets[0] = 0, non-decreasing
 *   ap_records      device or host, double [n_centres][8] or NULL, WRITTEN (not accumulated):
 *                   e1(a), e2(a), e4(a), e1(w), e2(w), e4(w), galaxies inside the cut, 0
 *   moments         device or host, double [n_theta][8]: entries 0..4 ACCUMULATED
 *                   (sum e4(a), sum e4(w), sum e2(a), sum e2(w), apertures), so patches add
 *                   up; entries 5..7 recomputed from them on every call:
 *                   <M_ap^4> = A^4 [0]/[1], <M_ap^2> = A^2 [2]/[3], A = pi (4 theta)^2 the
 *                   area of the cut disc, and the connected part <M_ap^4> - 3 <M_ap^2>^2.
 *                   Summing numerators and denominators weights each aperture's ratio by
 *                   its denominator (inverse shot-noise weights).
 * Device-only calls are stream-ordered after one synchronisation (the bounding box of the
 * catalogue is read back to size the grid); host outputs make the call synchronous.
 * Returns EXT4PCF_OK, EXT4PCF_E_INVALID_ARG, EXT4PCF_E_OOM or EXT4PCF_E_CUDA. */
EXT4PCF_API int ext4pcf_map_direct(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                                   const double* weights, int64_t n_gal, const double* thetas,
                                   int n_theta, const double* centres, const int64_t* centre_offsets,
                                   double* ap_records, double* moments);

/* Natural components of the shear N-point function (paper App. F.1).  The 2^{N-1} rows of
 * the sign matrix beta (beta[mu][l] = -1 where the l-th shear of Gamma_mu is complex
 * conjugated, else +1), in the paper's order: p = 0, 1, ..., floor(N/2) conjugated shears,
 * for each p the conjugated positions in lexicographic order, and for even N only the first
 * half of the p = N/2 rows (the others are their complex conjugates).  At N = 4 the rows are
 * the components Gamma_0 .. Gamma_7 of ext4pcf_measure.
 *   order  N, 2 .. 16
 *   beta   host, int [2^{N-1}][N], or NULL to query the count
 *   cap    ints available in beta
 * Host only (no device, no context).  Returns 2^{N-1}, or EXT4PCF_E_INVALID_ARG. */
EXT4PCF_API int ext4pcf_nth_order_components(int order, int* beta, int cap);

/* Multipole factorisation of component mu in the x-projection (paper App. F.2):
 *   Upsilon_{mu,n}(Theta_1 .. Theta_{N-1}) = sign * sum_i t_i * prod_{l=1}^{N-1} F_l(theta_i, Theta_l)
 * with n = (n_2 .. n_{N-1}); t_i = w_i gamma_c,i (centre code 0), w_i gamma_c,i^* (1) or w_i (2);
 * F_l = G_m, conj(G_m), or W_m for the normalisation (mu = -1), where
 * m = sum_k a_{l,k} n_k + b_l and G_m(theta_i, Theta) = sum_j w_j gamma_c,j e^{i m phi_ij}.
 *   order  N, 2 .. 16;  mu  0 .. 2^{N-1}-1, or -1 for the normalisation
 *   table  host, int, or NULL to query the size 2 + (N-1)(N+1):
 *          [0] sign (-1)^N (+1 for the normalisation), [1] centre code, then for
 *          l = 1 .. N-1 a row of N+1 ints: array (0 G, 1 W), conj (0/1), a_{l,2} .. a_{l,N-1}, b_l
 *   cap    ints available in table
 * Host only.  Returns the size, or EXT4PCF_E_INVALID_ARG. */
EXT4PCF_API int ext4pcf_nth_order_factors(int order, int mu, int* table, int cap);

/* Multipoles of the shear 3PCF, the order-3 case of the N-th order estimator (paper App. F).
 * The neighbour multipoles are gathered as for ext4pcf_measure, in FP64 when the context's
 * precision is EXT4PCF_FP64 and in FP32 (cell-anchored positions) for every other precision;
 * the contraction forms its products and sums in FP64 either way.  It reads
 * the tables of ext4pcf_nth_order_factors(3, mu), and when Theta1 = Theta2 it subtracts the
 * term in which both neighbours are the same galaxy, so that only triplets of distinct
 * galaxies remain:
 *   Upsilon_{mu,n}(Theta1, Theta2) = sign sum_{i, j != k} t_i F1_j F2_k  (mu = 0..3, natural
 *   components Gamma_0..3 in the order of ext4pcf_nth_order_components(3)), and the
 *   normalisation N_n = sum_{i, j != k} w_i w_j w_k e^{i n (phi_ij - phi_ik)}.
 *   positions, shears, weights  device, as for ext4pcf_measure (one catalogue)
 *   radial_bins  host [n_bins+1] as for ext4pcf_measure;  n_bins 1..32;  n_max 0..40, with the
 *                record limit of ext4pcf_measure (larger records: EXT4PCF_E_UNSUPPORTED)
 *   upsilon3     device, double [5][2 n_max + 1][n_bins][n_bins][2] (index 4 the
 *                normalisation; axes n + n_max, Theta1, Theta2), accumulated into
 * Stream-ordered, returns after enqueueing (see the conventions above).  Waves hold
 * ext4pcf_config.wave_centres centres (0: 4096).  Returns EXT4PCF_OK, EXT4PCF_E_INVALID_ARG
 * (including host pointers), EXT4PCF_E_OOM, EXT4PCF_E_CUDA, or EXT4PCF_E_UNSUPPORTED when a
 * factor index of the generated order-3 tables falls outside the gathered multipole range
 * for this n_max (checked before any work; no n_max in 0..40 does this today). */
EXT4PCF_API int ext4pcf_measure3(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                                 const double* weights, int64_t n_gal, const double* radial_bins,
                                 int n_bins, int n_max, double* upsilon3);

/* The factor tables compiled into the 4PCF contraction kernels, for inspection, in the
 * layout of ext4pcf_nth_order_factors at order 4 (row mu = 0..7, row 8 the normalisation;
 * 17 ints per row).
 *   which  0: CUDA-core contraction (FP64 / FP32 forms), 1: tensor-core contraction,
 *          2: the exchange of Theta2 and Theta3 used by the tensor-core contraction (Table
 *          tab:4PCFSymm): per component mu the pair (mu', o) with
 *          Upsilon_mu[n2, n3](Th1, Th2, Th3) = Upsilon_mu'[n3 + o, n2 - o](Th1, Th3, Th2),
 *          derived from the tensor-core factor table (18 ints)
 *   table  host, int [9][17] (which 0, 1) or [9][2] (which 2), or NULL to query the size;
 *   cap    ints available
 * Host only.  Returns 153 (18 for which = 2), or EXT4PCF_E_INVALID_ARG. */
EXT4PCF_API int ext4pcf_contraction_tables(int which, int* table, int cap);

/* Message of the last failure on this context ("" if none).  Valid until the next call. */
EXT4PCF_API const char* ext4pcf_last_error(const ext4pcf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* EXT4PCF_H */
