// Tensor-core contraction of a wave (tcgen05, sm_103a).
//
// For fixed s = n2 + n3 every natural component factorises as
//   Upsilon_mu[n2,n3](Th1,Th2,Th3) = sum_i A_i^mu[s](Th1) * KR_i[n2,n3](Th2,Th3),
//   KR_i = xt_i * B_i[n2](Th2) * C_i[n3](Th3)   (a Khatri-Rao product over the centre i),
// i.e. a complex GEMM over the centre index.  Components that share KR (mu = 0 and 2;
// mu = 1 and 5) share the GEMM.  Mapping onto tcgen05.mma (M = 128, K along centres):
//   * A operand (TMEM): 128 KR rows (n2, Th2 <= Th3) of one s.  Row r of the tile is TMEM
//     lane r; centre i occupies K elements (2i, 2i+1) = (re, im).  Sixteen producer warps
//     form KR on the CUDA cores and write it with tcgen05.st (warp w owns lanes
//     32 (w % 4) ..; the four warps of a lane group split the 32 centres of a stage).
//   * B operand (shared memory, K-major, 128-byte swizzle): column (mu, Th1, re|im) holds
//     the real embedding of A_i^mu(Th1): K rows (2i, 2i+1) = (Ar, -Ai) for the real output
//     and (Ai, Ar) for the imaginary output, so that D = A_op B_op is the complex product.
//   * D (TMEM, FP32): 128 rows x (2 * #mu * nb, padded to 16) columns.  Every 64 centres the
//     partial sum is promoted out of TMEM into FP32 registers (two D buffers alternate, so
//     the MMAs run on meanwhile); the long FP32 accumulation inside the tensor core would
//     otherwise lose bits.  The epilogue adds the sums into the FP64 reduced output.
// Staging: a pre-pass writes the wave's x~B values and G, W multipoles transposed (one row
// per (quantity, multipole, bin), the centres along the row); a loader warp copies each
// stage's rows (32 centres) into shared memory with 2D TMA boxes of 16 centres x 8 rows
// (128-byte swizzle, so that eight lanes reading eight rows hit different banks).
// Precision: BF16x3 splits every operand into bf16 hi + lo and accumulates
// hi*hi + hi*lo + lo*hi (kind::f16); 3xTF32 does the same with tf32 hi + lo (kind::tf32,
// ~22 mantissa bits per operand); TF32 uses one kind::tf32 pass.
// The split-FP16 form has a kernel of its own (contract_h16.cu) with the same work items and
// reduced output.
// Every wait is bounded by a clock budget; on expiry the kernel records an error code, runs
// to its end, waits for its own MMAs and copies and frees its TMEM.
//
// Symmetry reduction (Table tab:4PCFSymm, the column that swaps Theta2 and Theta3): for
// every component mu there is a component mu' and an offset o with
//   Upsilon_mu[n2, n3](Th1, Th2, Th3) = Upsilon_mu'[n3 + o, n2 - o](Th1, Th3, Th2).
// The tile rows therefore run over the bin pairs Th2 <= Th3 only (nb (nb + 1) / 2 of nb^2),
// and over the multipoles the map reaches from |n2|, |n3| <= N (one more n2 per s); the
// results go to a reduced FP64 array [9][2N+3][2N+3][nb][pairs], from which tc_expand adds
// every ordered triple at |n| <= N into the output once per catalogue.  mu' and o are derived
// on the host from the factor table below (derive_swap_map), not typed in.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kr_table.cuh"
#include "tc_ptx.cuh"

namespace ext4pcf {

namespace {

constexpr int kStageCentres = 32;
constexpr int kProducerWarps = 16;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 64;  // + the MMA issuer warp and the TMA loader warp
constexpr uint32_t kTmemCols = 512;
constexpr int kDCols = 128;          // D region: two 64-column buffers
constexpr int kMaxNpad = 64;         // B columns: 2 * #mu * nb padded to 16 (nb <= 16)

// bf16 hi/lo split of a pair (re, im) packed as bf16x2 (re in the low half)
__device__ __forceinline__ void split_bf16(float re, float im, uint32_t& hi, uint32_t& lo) {
  uint32_t h;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(im), "f"(re));
  const float hr = __uint_as_float(h << 16), hi_ = __uint_as_float(h & 0xFFFF0000u);
  uint32_t l;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(im - hi_), "f"(re - hr));
  hi = h;
  lo = l;
}

struct TcArgs {
  Layout L;
  int T;              // centres of the wave at most
  const int* n_live;  // with w0: the wave's centres on the device (wave_centres)
  int w0;
  double* red;        // reduced output [9][2N+3][2N+3][nb][npairs] (complex, FP64)
  int npairs;         // nb (nb + 1) / 2
  const int4* items;  // (type, s, row0, nrows | (n2 of row 0 of the s block + 64) << 8)
  int n_items;
  int row_g, row_w;   // first row of G and of W in the transposed wave array (x~B rows from 0)
  int in_stages;      // depth of the staged-input ring
  int stage_rows;     // rows per staged stage and half (multiple of 8)
  long long timeout;
  int* status;
};

// The transposed wave array (one row per (quantity, multipole, bin), the wave's centres along
// the row, padded to a multiple of 32):
//   rows [0, row_g)       x~ B per row type of B: (xb type, n2 + N + 1, bin), n2 in [-N-1, N+1]
//   rows [row_g, row_w)   G_n(bin), n in [-2N-3, 2N-1]
//   rows [row_w, rows)    W_m(bin), m in [0, 2N]
// x~ B: 0: x G[-n2-2]   1: x G[n2-2]^*   2: x^* G[-n2-2]   3: x^* G[n2-2]^*   4: w W[-n2] (|n2| <= N)

__device__ __forceinline__ float2 wave_value(const Layout& L, const float2* __restrict__ rc, float2 x, float w,
                                             int r, int row_g, int row_w) {
  const int nb = L.nb, N = L.N, nx = 2 * N + 3;
  if (r >= row_w) return rc[L.oW + (r - row_w)];
  if (r >= row_g) return rc[L.oG + (r - row_g)];
  const int t = r / (nx * nb), n2 = (r / nb) % nx - N - 1, b = r % nb;
  float2 f;
  if (t == 4) {
    // the normalisation rows keep |n2| <= N (its swap partner is itself, o = 0)
    const int m = -n2;
    f = (m <= N && m >= -N) ? rc[L.W(m >= 0 ? m : -m, b)] : make_float2(0.f, 0.f);
    if (m < 0) f.y = -f.y;
    x = make_float2(w, 0.f);
  } else {
    f = (t & 1) ? rc[L.G(n2 - 2, b)] : rc[L.G(-n2 - 2, b)];
    if (t & 1) f.y = -f.y;
    if (t >= 2) x.y = -x.y;
  }
  return make_float2(x.x * f.x - x.y * f.y, x.x * f.y + x.y * f.x);
}

// 32 rows x 32 centres per block through shared memory: reads along each centre's record,
// writes along the centres of each row (both coalesced)
// Centres from the wave's count up to the next multiple of 32 are written as zeros (the last
// stage of the contraction reads them); columns beyond are never read.
__global__ void __launch_bounds__(256) transpose_wave_kernel(const Layout L, const float2* __restrict__ rec,
                                                             const float2* __restrict__ xw, int T,
                                                             const int* __restrict__ n_live, int w0, int Tp,
                                                             int row_g, int row_w, int rows,
                                                             float2* __restrict__ out) {
  __shared__ float2 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  T = wave_centres(T, n_live, w0);
  if (c0 >= T) return;  // whole column tiles past the wave (uniform per block)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + ty + 8 * k, r = r0 + tx;
    float2 v = make_float2(0.f, 0.f);
    if (c < T && r < rows)
      v = wave_value(L, rec + (size_t)c * L.rec, xw[2 * (size_t)c], xw[2 * (size_t)c + 1].x, r, row_g, row_w);
    tile[ty + 8 * k][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    if (r < rows && c < Tp) out[(size_t)r * Tp + c] = tile[tx][ty + 8 * k];
  }
}

// Rows of the transposed array holding factor f for its variable in [va, vb]; `lo` is the
// first multipole index (n for G, m = |n| for W).
struct RowBlk {
  int row0, len, lo, is_w;
};
__device__ __forceinline__ RowBlk row_blk(const TcArgs& a, KF f, int va, int vb) {
  const int nb = a.L.nb, N = a.L.N;
  const int nlo = f.sgn > 0 ? va + f.off : -vb + f.off;
  const int nhi = f.sgn > 0 ? vb + f.off : -va + f.off;
  RowBlk b;
  b.is_w = f.arr;
  if (f.arr == 0) {
    b.lo = nlo;
    b.row0 = a.row_g + (nlo + 2 * N + 3) * nb;
    b.len = (nhi - nlo + 1) * nb;
  } else {
    int mlo, mhi;
    if (nlo >= 0) { mlo = nlo; mhi = nhi; }
    else if (nhi <= 0) { mlo = -nhi; mhi = -nlo; }
    else { mlo = 0; mhi = max(-nlo, nhi); }
    b.lo = mlo;
    b.row0 = a.row_w + mlo * nb;
    b.len = (mhi - mlo + 1) * nb;
  }
  return b;
}
// row (within the block) and conjugation of factor f at variable v, bin b
__device__ __forceinline__ int blk_index(const RowBlk& k, KF f, int v, int b, int nb, bool& cj) {
  const int n = f.sgn * v + f.off;
  cj = f.conj != 0;
  if (!k.is_w) return (n - k.lo) * nb + b;
  cj ^= (n < 0);
  return ((n < 0 ? -n : n) - k.lo) * nb + b;
}

// Geometry of one work item: the staged blocks (x~B rows, C rows, A rows) of every stage and
// their rows in the staged buffer (each block starts at a multiple of 8 rows: one TMA box).
struct ItemGeo {
  int type, s, row0, nrows, n2a, t2a, t2b;
  RowBlk bx, bc, ba0, ba1;
  int sx, sc, sa0, sa1;
};
__device__ __forceinline__ int round8(int v) { return (v + 7) & ~7; }
__device__ __forceinline__ ItemGeo item_geo(const TcArgs& a, int4 item, const KRType& kr) {
  const int nb = a.L.nb, N = a.L.N, nx = 2 * N + 3;
  ItemGeo g;
  g.type = item.x;
  g.s = item.y;
  g.row0 = item.z;
  g.nrows = item.w & 0xFF;
  g.n2a = (item.w >> 8) - 64;
  g.t2a = g.n2a + g.row0 / a.npairs;
  g.t2b = g.n2a + (g.row0 + g.nrows - 1) / a.npairs;
  g.bx.row0 = (kXBOfType[g.type] * nx + (g.t2a + N + 1)) * nb;
  g.bx.len = (g.t2b - g.t2a + 1) * nb;
  g.bx.lo = g.t2a;
  g.bx.is_w = 0;
  g.bc = row_blk(a, kr.C, g.s - g.t2b, g.s - g.t2a);
  g.ba0 = row_blk(a, kr.A[0], g.s, g.s);
  g.ba1 = kr.nmu > 1 ? row_blk(a, kr.A[1], g.s, g.s) : RowBlk{0, 0, 0, 0};
  g.sx = 0;
  g.sc = round8(g.bx.len);
  g.sa0 = g.sc + round8(g.bc.len);
  g.sa1 = g.sa0 + round8(g.ba0.len);
  return g;
}

// byte offset, inside one half of a staged stage, of the 16-byte chunk c of row e (the TMA's
// 128-byte swizzle: chunk index XOR row mod 8)
__device__ __forceinline__ uint32_t stg_off(int e, int c) { return (uint32_t)(e * 128 + ((c ^ (e & 7)) << 4)); }

// stages per TMEM partial sum (64 centres): the tensor core's FP32 accumulation loses bits
// in proportion to the MMAs it accumulates (measured: ~3e-4 over 750 MMAs, ~5e-5 over
// 96, ~1.5e-4 over 192 for 3xTF32), so partial sums are short and summed in registers
constexpr int kPromote = 2;
constexpr int kDBuf = 64;    // two D buffers of 64 columns (npad <= 64)
constexpr int kQuarter = kStageCentres / (kProducerWarps / 4);  // centres per producer warp
constexpr int kWarpMma = kProducerWarps, kWarpLoad = kProducerWarps + 1;
constexpr int kBoxRows = 8;     // rows per TMA box
constexpr int kMaxInStages = 4; // staged-input ring depth (at most)

// Per precision: stages, TMEM columns and 128-byte-wide shared-memory K-atoms per stage.
template <int PREC> struct TcPrec;
template <> struct TcPrec<EXT4PCF_SPLIT_BF16> {  // A: hi | lo (bf16x2); B: hi atom | lo atom
  static constexpr int kStages = 4, kStageCols = 64, kAtoms = 2;
};
template <> struct TcPrec<EXT4PCF_TF32> {  // A: fp32 (re, im) pairs; B: two atoms
  static constexpr int kStages = 4, kStageCols = 64, kAtoms = 2;
};
template <> struct TcPrec<EXT4PCF_3XTF32> {  // A: hi | lo fp32 pairs; B: hi 2 atoms | lo 2 atoms
  static constexpr int kStages = 3, kStageCols = 128, kAtoms = 4;
};

// Warp roles: warps 0..15 form the A operand (Khatri-Rao rows, TMEM) and the B operand
// (shared memory) of each stage; warp 16 issues the MMAs (one thread); warp 17 stages each
// stage's rows of the transposed wave array with TMA (one thread).  Rings and their
// mbarriers (counts in brackets):
//   staged input  in_full [1 + TMA bytes] / in_empty [16 producer warps]
//   A and B       ab_full [16 producer warps] / ab_empty [1, tcgen05.commit]
//   partial sums  dfull [1, tcgen05.commit] / dempty [16 producer warps]
// Producer warps run on their own: a warp waits only for its stage's data and for a free
// A/B slot, and arrives once per stage (lane 0, after __syncwarp).
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
contract_tc_kernel(const TcArgs args, const __grid_constant__ CUtensorMap tmap) {
  using P = TcPrec<PREC>;
  // kind::f16 operands: bf16 halves, one 32-bit word per centre (re, im)
  constexpr bool k16 = PREC == EXT4PCF_SPLIT_BF16;
  constexpr int kSt = P::kStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const Layout L = args.L;
  const int nb = L.nb, N = L.N, npairs = args.npairs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int tile_bytes = kMaxNpad * 128;  // one 128-byte-wide K-atom (npad <= 64)
  constexpr int stage_bytes = P::kAtoms * tile_bytes;
  const int S_in = args.in_stages;
  const uint32_t half_bytes = (uint32_t)args.stage_rows * 128u;
  unsigned char* in_base = sm + kSt * stage_bytes;  // S_in stages of two halves
  uint64_t* bars = reinterpret_cast<uint64_t*>(in_base + (size_t)S_in * 2 * half_bytes);
  uint64_t* in_full = bars;
  uint64_t* in_empty = in_full + kMaxInStages;
  uint64_t* ab_full = in_empty + kMaxInStages;
  uint64_t* ab_empty = ab_full + kSt;
  uint64_t* dfull = ab_empty + kSt;  // [2]
  uint64_t* dempty = dfull + 2;      // [2]
  uint64_t* drain = dempty + 2;      // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int k = 0; k < S_in; ++k) {
      mbar_init(&in_full[k], 1);
      mbar_init(&in_empty[k], kProducerWarps);
    }
    for (int k = 0; k < kSt; ++k) {
      mbar_init(&ab_full[k], kProducerWarps);
      mbar_init(&ab_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&dfull[k], 1);
      mbar_init(&dempty[k], kProducerWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kWarpLoad && lane == 0) tma_prefetch_desc(&tmap);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long budget = args.timeout;
  const int nstage = (wave_centres(args.T, args.n_live, args.w0) + kStageCentres - 1) / kStageCentres;
  const int nsub = (nstage + kPromote - 1) / kPromote;
  int err = 0;
  // bounded wait on an mbarrier phase; the first wait of the CTA that runs out of its budget
  // raises the abort flag, after which every wait gives up at once, so that a broken
  // pipeline ends the kernel quickly (with the status word set) instead of waiting out the
  // budget at every stage
  auto wait = [&](uint64_t* b, uint32_t parity) -> bool {
    if (*abort_flag) {
      err = 1;
      return false;
    }
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity)) {
      if (*abort_flag || clock64() - t0 > budget) {
        *abort_flag = 1;
        err = 1;
        return false;
      }
    }
    return true;
  };

  if (warp < kProducerWarps) {
    // ---------------------------------------------------------------------- producers
    const int grp = warp & 3, quarter = warp >> 2;
    const int h = quarter >> 1, c0 = (quarter & 1) * 4;  // half and first 16-byte chunk of my centres
    long long qi = 0, qa = 0, gs = 0;                    // input stages, A/B stages, partial sums
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const KRType kr = kKR[args.items[it].x];
      const ItemGeo g = item_geo(args, args.items[it], kr);
      const int nmu = kr.nmu, ncols = 2 * nmu * nb;
      const int rl = grp * 32 + lane;  // tile row = TMEM lane
      const bool row_ok = rl < g.nrows;
      const int rr = g.row0 + (row_ok ? rl : 0);
      const int n2 = g.n2a + rr / npairs, n3 = g.s - n2;
      int b2, b3;
      pair_of(rr % npairs, nb, b2, b3);
      bool cjC;
      const int eB = g.sx + (n2 - g.t2a) * nb + b2;
      const int eC = g.sc + blk_index(g.bc, kr.C, n3, b3, nb, cjC);
      const float sgnC = cjC ? -1.f : 1.f;
      // byte offsets (inside a staged stage) of the four 16-byte chunks (two centres each) of
      // this warp's eight centres in this row's x~B and C slots
      uint32_t offB[4], offC[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        offB[q] = (uint32_t)h * half_bytes + stg_off(eB, c0 + q);
        offC[q] = (uint32_t)h * half_bytes + stg_off(eC, c0 + q);
      }
      // this warp's column pairs v = (component slot, Th1) of the B operand (at most two, as
      // nmu nb <= 32 for the supported shapes), with their staged row and conjugation, fixed
      // for the item: kept in registers (no runtime-indexed access to the factor tables)
      const int nv = nmu * nb;
      int eAv[2] = {0, 0};
      bool cjAv[2] = {false, false};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int v = warp + j * kProducerWarps;
        if (v < nv) {
          const int b1 = v % nb;
          if (v < nb) eAv[j] = g.sa0 + blk_index(g.ba0, kr.A[0], g.s, b1, nb, cjAv[j]);
          else eAv[j] = g.sa1 + blk_index(g.ba1, kr.A[1], g.s, b1, nb, cjAv[j]);
        }
      }
      const int mu0 = kr.mu[0], mu1 = kr.mu[1];
      // shared-memory offsets of this lane's centre: the A value in the staged stage, and the
      // words of the two B columns (re, im) in the B tile
      uint32_t aoff[2], bre[2], bim[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int v = warp + j * kProducerWarps;
        aoff[j] = (uint32_t)(lane >> 4) * half_bytes + stg_off(eAv[j], (lane & 15) >> 1) + (lane & 1) * 8;
        const int kw = k16 ? lane : 2 * lane;  // K word of the centre
        bre[j] = sw128_word_off(2 * v, kw, kMaxNpad);
        bim[j] = sw128_word_off(2 * v + 1, kw, kMaxNpad);
      }
      float accD[16];  // FP32 sums of the promoted partials: this row, 16 columns
#pragma unroll
      for (int j = 0; j < 16; ++j) accD[j] = 0.f;
      auto promote = [&](long long gg) {  // read partial sum gg from its D buffer
        const int buf = (int)(gg & 1);
        wait(&dfull[buf], (uint32_t)((gg >> 1) & 1));
        tc_fence_after();
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(grp * 32) << 16) + buf * kDBuf + quarter * 16, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) accD[j] += __uint_as_float(v[j]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dempty[buf]);
      };
      const long long gs0 = gs;
      for (int k = 0; k < nstage; ++k, ++qi, ++qa) {
        const int islot = (int)(qi % S_in), aslot = (int)(qa % kSt);
        wait(&in_full[islot], (uint32_t)((qi / S_in) & 1));
        wait(&ab_empty[aslot], (uint32_t)(((qa / kSt) & 1) ^ 1));
        tc_fence_after();
        const unsigned char* st = in_base + (size_t)islot * 2 * half_bytes;
        unsigned char* bt = sm + aslot * stage_bytes;
        // B operand (shared memory, K-major, swizzled): the real embedding of A(Th1) for the
        // 32 centres of the stage; warp v forms column pair v = (g, b1), lane = centre
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (warp + j * kProducerWarps >= nv) break;
          float2 a = *reinterpret_cast<const float2*>(st + aoff[j]);
          if (cjAv[j]) a.y = -a.y;
          if (PREC == EXT4PCF_SPLIT_BF16) {
            uint32_t rh, rl, ih, il;  // column re: (Ar, -Ai), column im: (Ai, Ar), bf16x2 each
            split_bf16(a.x, -a.y, rh, rl);
            split_bf16(a.y, a.x, ih, il);
            *reinterpret_cast<uint32_t*>(bt + bre[j]) = rh;
            *reinterpret_cast<uint32_t*>(bt + tile_bytes + bre[j]) = rl;
            *reinterpret_cast<uint32_t*>(bt + bim[j]) = ih;
            *reinterpret_cast<uint32_t*>(bt + tile_bytes + bim[j]) = il;
          } else if (PREC == EXT4PCF_TF32) {
            *reinterpret_cast<float2*>(bt + bre[j]) = make_float2(a.x, -a.y);
            *reinterpret_cast<float2*>(bt + bim[j]) = make_float2(a.y, a.x);
          } else {
            uint32_t xh, xl, yh, yl;
            split_tf32(a.x, xh, xl);
            split_tf32(a.y, yh, yl);
            const uint32_t sgn = 0x80000000u;
            *reinterpret_cast<uint2*>(bt + bre[j]) = make_uint2(xh, yh ^ sgn);
            *reinterpret_cast<uint2*>(bt + bim[j]) = make_uint2(yh, xh);
            *reinterpret_cast<uint2*>(bt + 2 * tile_bytes + bre[j]) = make_uint2(xl, yl ^ sgn);
            *reinterpret_cast<uint2*>(bt + 2 * tile_bytes + bim[j]) = make_uint2(yl, xl);
          }
        }
        // A operand (TMEM): this row's Khatri-Rao values x~B * C for the warp's eight centres
        float2 xbv[kQuarter], cvv[kQuarter];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 tb = *reinterpret_cast<const float4*>(st + offB[q]);
          const float4 tc = *reinterpret_cast<const float4*>(st + offC[q]);
          xbv[2 * q] = make_float2(tb.x, tb.y);
          xbv[2 * q + 1] = make_float2(tb.z, tb.w);
          cvv[2 * q] = make_float2(tc.x, tc.y);
          cvv[2 * q + 1] = make_float2(tc.z, tc.w);
        }
        const uint32_t acol = tmem + ((uint32_t)(grp * 32) << 16) + kDCols + aslot * P::kStageCols;
        if (PREC == EXT4PCF_SPLIT_BF16) {
          uint32_t w[16];
#pragma unroll
          for (int j = 0; j < kQuarter; ++j) {
            const float2 xb = xbv[j];
            float2 cv = cvv[j];
            cv.y *= sgnC;
            split_bf16(xb.x * cv.x - xb.y * cv.y, xb.x * cv.y + xb.y * cv.x, w[j], w[8 + j]);
          }
          tmem_st8(acol + quarter * 8, w);
          tmem_st8(acol + 32 + quarter * 8, w + 8);
        } else if (PREC == EXT4PCF_TF32) {
          uint32_t w[16];
#pragma unroll
          for (int j = 0; j < kQuarter; ++j) {
            const float2 xb = xbv[j];
            float2 cv = cvv[j];
            cv.y *= sgnC;
            w[2 * j] = __float_as_uint(xb.x * cv.x - xb.y * cv.y);
            w[2 * j + 1] = __float_as_uint(xb.x * cv.y + xb.y * cv.x);
          }
          tmem_st16(acol + quarter * 16, w);
        } else {
          uint32_t wh[16], wl[16];
#pragma unroll
          for (int j = 0; j < kQuarter; ++j) {
            const float2 xb = xbv[j];
            float2 cv = cvv[j];
            cv.y *= sgnC;
            split_tf32(xb.x * cv.x - xb.y * cv.y, wh[2 * j], wl[2 * j]);
            split_tf32(xb.x * cv.y + xb.y * cv.x, wh[2 * j + 1], wl[2 * j + 1]);
          }
          tmem_st16(acol + quarter * 16, wh);
          tmem_st16(acol + 64 + quarter * 16, wl);
        }
        // every value this warp loaded from the staged input has been used (the stores above
        // read the products): the staged stage can be refilled
        __syncwarp();
        if (lane == 0) mbar_arrive(&in_empty[islot]);
        tmem_wait_st();
        fence_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ab_full[aslot]);
        // a partial sum finished one promotion block ago is read while the MMAs run on
        if ((k % kPromote) == kPromote - 1 && k / kPromote >= 1) promote(gs0 + k / kPromote - 1);
      }
      // the remaining partial sums of this item: the loop read partials 0 .. F-2
      // (F = complete promotion blocks)
      const int read_in_loop = max(0, nstage / kPromote - 1);
      for (long long gg = gs0 + read_in_loop; gg < gs0 + nsub; ++gg) promote(gg);
      gs = gs0 + nsub;
      // ---------------------------------------------------------------- epilogue
      if (row_ok && nstage > 0) {  // (a wave past the end adds nothing)
        const int pr = rr % npairs, nx = 2 * N + 3;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int n = quarter * 16 + j;
          if (n < ncols) {
            const int ga = n / (2 * nb), b1 = (n >> 1) % nb;
            const int mu = ga ? mu1 : mu0;
            const size_t o = ((((size_t)mu * nx + (n2 + N + 1)) * nx + (n3 + N + 1)) * nb + b1) * npairs + pr;
            double* p = args.red + 2 * o;
            p[0] += (double)accD[j];
            p[1] += (double)accD[j + 1];
          }
        }
      }
    }
  } else if (warp == kWarpMma) {
    // ---------------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint64_t dbase = desc_sw128(saddr(sm));
      long long qa = 0, gs = 0;
      for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
        const KRType kr = kKR[args.items[it].x];
        const int npad = (2 * kr.nmu * nb + 15) / 16 * 16;
        const uint32_t id = PREC == EXT4PCF_SPLIT_BF16 ? idesc(1u, npad) : idesc(2u, npad);
        for (int k = 0; k < nstage; ++k, ++qa) {
          const long long gg = gs + k / kPromote;
          const int buf = (int)(gg & 1);
          const bool first = (k % kPromote) == 0;
          if (first && gg >= 2) {
            wait(&dempty[buf], (uint32_t)(((gg >> 1) - 1) & 1));
          }
          const int slot = (int)(qa % kSt);
          wait(&ab_full[slot], (uint32_t)((qa / kSt) & 1));
          tc_fence_after();
          const uint32_t d = tmem + buf * kDBuf;
          const uint32_t a0 = tmem + kDCols + slot * P::kStageCols;
          // descriptor of the slot's B tile: the start-address field (bits 0-13, address / 16)
          // of the first tile's descriptor plus the offset / 16 (no carry: shared addresses
          // stay below 2^18)
          const uint64_t db = dbase + (uint64_t)((slot * stage_bytes) >> 4);
          if (k16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // K = 16 halves = 8 centres per MMA
              const uint64_t bh = db + (q * 32 >> 4), bl = db + ((tile_bytes + q * 32) >> 4);
              mma_f16(d, a0 + q * 8, bh, id, (!first || q > 0) ? 1u : 0u);
              mma_f16(d, a0 + q * 8, bl, id, 1u);
              mma_f16(d, a0 + 32 + q * 8, bh, id, 1u);
            }
          } else if (PREC == EXT4PCF_TF32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // K = 8 fp32 = 4 centres per MMA
              const uint64_t b = db + (((q >> 2) * tile_bytes + (q & 3) * 32) >> 4);
              mma_tf32(d, a0 + q * 8, b, id, (!first || q > 0) ? 1u : 0u);
            }
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // hi*hi + hi*lo + lo*hi, K = 8 fp32 per MMA
              const uint32_t bo_ = (q >> 2) * tile_bytes + (q & 3) * 32;
              const uint64_t bh = db + (bo_ >> 4), bl = db + ((2 * tile_bytes + bo_) >> 4);
              mma_tf32(d, a0 + q * 8, bh, id, (!first || q > 0) ? 1u : 0u);
              mma_tf32(d, a0 + q * 8, bl, id, 1u);
              mma_tf32(d, a0 + 64 + q * 8, bh, id, 1u);
            }
          }
          mma_commit(&ab_empty[slot]);
          if ((k % kPromote) == kPromote - 1 || k == nstage - 1) mma_commit(&dfull[buf]);
        }
        gs += nsub;
      }
      // every MMA of this CTA has completed before the TMEM is released (also when a wait
      // above gave up); an MMA always finishes, so this bound is generous
      mma_commit(drain);
      if (!mbar_wait(drain, 0u, 4000000000LL)) err = 1;
    }
    __syncwarp();
  } else if (warp == kWarpLoad) {
    // ---------------------------------------------------------------------- TMA loader
    if (lane == 0) {
      long long qi = 0;
      long long last[kMaxInStages];  // last stage whose copies were issued, per slot
      for (int k = 0; k < kMaxInStages; ++k) last[k] = -1;
      for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
        const KRType kr = kKR[args.items[it].x];
        const ItemGeo g = item_geo(args, args.items[it], kr);
        const RowBlk blk[4] = {g.bx, g.bc, g.ba0, g.ba1};
        const int srow[4] = {g.sx, g.sc, g.sa0, g.sa1};
        if (g.sa1 + round8(g.ba1.len) > args.stage_rows) {  // never for the supported shapes
          *abort_flag = 1;
          err = 1;
        }
        uint32_t boxes = 0;
        for (int b = 0; b < 4; ++b) boxes += (uint32_t)((blk[b].len + kBoxRows - 1) / kBoxRows);
        const uint32_t bytes = boxes * 2u * kBoxRows * 128u;
        for (int k = 0; k < nstage; ++k, ++qi) {
          const int islot = (int)(qi % S_in);
          wait(&in_empty[islot], (uint32_t)(((qi / S_in) & 1) ^ 1));
          if (*abort_flag) continue;  // nothing more is copied once the CTA gives up
          last[islot] = qi;
          mbar_expect_tx(&in_full[islot], bytes);
          unsigned char* st = in_base + (size_t)islot * 2 * half_bytes;
          for (int b = 0; b < 4; ++b)
            for (int r = 0; r < blk[b].len; r += kBoxRows)
              for (int hh = 0; hh < 2; ++hh)
                tma_load_2d(st + hh * half_bytes + (srow[b] + r) * 128, &tmap, k * kStageCentres + hh * 16,
                            blk[b].row0 + r, &in_full[islot]);
        }
      }
      // every copy has landed before the shared memory is given up: the phases of a slot
      // complete in order, so its last issued phase covers the earlier ones (copies always
      // complete; the bound only guards against the unforeseen)
      for (int k = 0; k < S_in; ++k)
        if (last[k] >= 0 && !mbar_wait(&in_full[k], (uint32_t)((last[k] / S_in) & 1), 4000000000LL)) err = 1;
    }
    __syncwarp();
  }
  if (err) atomicExch(args.status, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// rows per staged stage and half: the x~B and C blocks of at most the tile's n2 values
// (128 rows = 128 / pairs values of n2, +2 for misalignment, at most 2N+3) and two A blocks,
// each rounded up to whole TMA boxes
int stage_rows_for(int nb, int N) {
  int rows = 128 / (nb * (nb + 1) / 2) + 2;
  if (rows > 2 * N + 3) rows = 2 * N + 3;
  auto r8 = [](int v) { return (v + 7) & ~7; };
  return 2 * r8(rows * nb) + 2 * r8(nb);
}

size_t tc_fixed_smem(int prec) {
  const bool x3 = prec == EXT4PCF_3XTF32;  // the others: 4 stages of 2 atoms
  const int st = x3 ? TcPrec<EXT4PCF_3XTF32>::kStages : 4;
  const int atoms = x3 ? TcPrec<EXT4PCF_3XTF32>::kAtoms : 2;
  return (size_t)st * atoms * kMaxNpad * 128 + 1024 + 512;
}

// staged-input ring depth that fits next to the B ring (0 if fewer than two stages fit)
int tc_in_stages(int nb, int N, int prec) {
  const size_t per = (size_t)stage_rows_for(nb, N) * 256;
  const size_t room = 227 * 1024 - tc_fixed_smem(prec);
  int k = (int)(room / per);
  if (k > kMaxInStages) k = kMaxInStages;
  return k >= 2 ? k : 0;
}

size_t tc_smem_bytes(int nb, int N, int prec) {
  return tc_fixed_smem(prec) + (size_t)tc_in_stages(nb, N, prec) * stage_rows_for(nb, N) * 256;
}

template <int PREC>
cudaError_t launch_tc(const TcArgs& a, const CUtensorMap& tm, size_t smem, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contract_tc_kernel<PREC><<<sms, kThreads, smem, s>>>(a, tm);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Layout& L, int precision) {
  if (precision == EXT4PCF_SPLIT_F16) return h16_supported(L);
  if (precision != EXT4PCF_SPLIT_BF16 && precision != EXT4PCF_TF32 && precision != EXT4PCF_3XTF32) return false;
  return L.nb >= 1 && 4 * L.nb <= kMaxNpad && tc_in_stages(L.nb, L.N, precision) >= 2;
}

// Work items of the reduced contraction: for every row type t and s = n2 + n3 the rows
// (n2, Th2 <= Th3) with n2 over the identity range max(-N, s-N) .. min(N, s+N), widened by one
// at the top (o = +1) or the bottom (o = -1) for the multipoles that the swap map reaches.
bool tc_build_items(const Layout& L, std::vector<int4>& items) {
  items.clear();
  signed char mup[9], off[9];
  if (!derive_swap_map(mup, off)) return false;
  const int N = L.N, npairs = L.nb * (L.nb + 1) / 2;
  for (int t = 0; t < kKRTypes; ++t) {
    const int o = type_offset(t, off);
    if (o < -1 || o > 1) return false;
    for (int s = -2 * N; s <= 2 * N; ++s) {
      int lo = s - N > -N ? s - N : -N, hi = s + N < N ? s + N : N;
      if (o > 0) ++hi;
      if (o < 0) --lo;
      const int rows = (hi - lo + 1) * npairs;
      for (int r0 = 0; r0 < rows; r0 += 128)
        items.push_back(make_int4(t, s, r0, (rows - r0 < 128 ? rows - r0 : 128) | ((lo + 64) << 8)));
    }
  }
  return true;
}

// rows of the transposed wave array (x~B, G, W) and its row pitch in centres
int tc_wave_rows(const Layout& L) { return (kXBTypes * (2 * L.N + 3) + L.nG + L.nW) * L.nb; }
int tc_wave_pitch(int T) { return (T + 31) / 32 * 32; }

size_t contract_tc_xb_bytes(const Layout& L, int T, int precision) {
  if (precision == EXT4PCF_SPLIT_F16) return contract_h16_wave_bytes(L, T);
  return (size_t)tc_wave_rows(L) * tc_wave_pitch(T) * sizeof(float2);
}


size_t tc_reduced_doubles(const Layout& L) {
  const size_t nx = 2 * L.N + 3;
  return (size_t)2 * 9 * nx * nx * L.nb * (L.nb * (L.nb + 1) / 2);
}

namespace {
struct SwapArgs {
  signed char mup[9], off[9];
};
// Every ordered triple at |n2|, |n3| <= N from the reduced array: Th2 <= Th3 directly, the
// others through the swap map.  One thread per output complex value, accumulated into ups.
__global__ void tc_expand_kernel(const Layout L, const SwapArgs sw, const double* __restrict__ red,
                                 double* __restrict__ ups) {
  const int N = L.N, nb = L.nb, nn = 2 * N + 1, nx = 2 * N + 3, npairs = nb * (nb + 1) / 2;
  const size_t nb3 = (size_t)nb * nb * nb, total = (size_t)9 * nn * nn * nb3;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b3 = (int)(e % nb), b2 = (int)((e / nb) % nb), b1 = (int)((e / ((size_t)nb * nb)) % nb);
    const size_t r = e / nb3;
    const int n3 = (int)(r % nn) - N, n2 = (int)((r / nn) % nn) - N, mu = (int)(r / ((size_t)nn * nn));
    int m = mu, m2 = n2, m3 = n3, p2 = b2, p3 = b3;
    if (b2 > b3) {
      m = sw.mup[mu];
      m2 = n3 + sw.off[mu];
      m3 = n2 - sw.off[mu];
      p2 = b3;
      p3 = b2;
    }
    const int pr = p2 * nb - p2 * (p2 - 1) / 2 + (p3 - p2);
    const size_t o = ((((size_t)m * nx + (m2 + N + 1)) * nx + (m3 + N + 1)) * nb + b1) * npairs + pr;
    ups[2 * e] += red[2 * o];
    ups[2 * e + 1] += red[2 * o + 1];
  }
}
}  // namespace

cudaError_t tc_expand(const Layout& L, const double* red, double* ups, cudaStream_t s) {
  SwapArgs sw;
  if (!derive_swap_map(sw.mup, sw.off)) return cudaErrorInvalidValue;
  const int nn = 2 * L.N + 1;
  const size_t total = (size_t)9 * nn * nn * L.nb * L.nb * L.nb;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 65536);
  tc_expand_kernel<<<blocks, 256, 0, s>>>(L, sw, red, ups);
  ++g_launches;
  return cudaGetLastError();
}

// mu' and o of every component (ext4pcf_contraction_tables, which = 2): 18 ints
int contraction_swap_map(int* out) {
  signed char mup[9], off[9];
  if (!derive_swap_map(mup, off)) return EXT4PCF_E_UNSUPPORTED;
  for (int mu = 0; mu < 9; ++mu) {
    out[2 * mu] = mup[mu];
    out[2 * mu + 1] = off[mu];
  }
  return 18;
}

namespace {
// cuTensorMapEncodeTiled from the driver, found once through the runtime (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}
}  // namespace

// 2D tensor map of a wave array of 8-byte elements: x elements per row (row_bytes apart), `rows`
// rows, boxes of 16 x 8 elements with the 128-byte swizzle
cudaError_t encode_wave_tmap(CUtensorMap* tm, const void* base, uint64_t x, uint64_t rows, uint64_t row_bytes) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)x, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {16, 8};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t contract_wave_tc(const Layout& L, const float2* rec, const float2* xw, int T, const int* n_live,
                             int w0, double* red, int precision, const int4* items, int n_items, float2* wave,
                             unsigned* rowmax, int* status, long long timeout, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  const int rows = tc_wave_rows(L), pitch = tc_wave_pitch(T);
  const int row_g = kXBTypes * (2 * L.N + 3) * L.nb, row_w = row_g + L.nG * L.nb;
  {
    dim3 grid((rows + 31) / 32, (T + 31) / 32);
    transpose_wave_kernel<<<grid, 256, 0, s>>>(L, rec, xw, T, n_live, w0, pitch, row_g, row_w, rows, wave);
    ++g_launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // 2D view: x = centre (T of them, pitch elements per row), y = row; boxes of 16 centres
  // (128 bytes, the swizzle span) by 8 rows; centres past T read as zero
  CUtensorMap tm;
  {
    cudaError_t e = encode_wave_tmap(&tm, wave, (uint64_t)T, (uint64_t)rows, (uint64_t)pitch * sizeof(float2));
    if (e != cudaSuccess) return e;
  }
  TcArgs a;
  a.L = L; a.T = T; a.n_live = n_live; a.w0 = w0; a.red = red;
  a.npairs = L.nb * (L.nb + 1) / 2;
  a.items = items; a.n_items = n_items;
  a.row_g = row_g; a.row_w = row_w;
  a.in_stages = tc_in_stages(L.nb, L.N, precision);
  a.stage_rows = stage_rows_for(L.nb, L.N);
  a.timeout = timeout; a.status = status;
  if (a.in_stages < 2) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = tc_smem_bytes(L.nb, L.N, precision);
  cudaError_t e;
  if (precision == EXT4PCF_SPLIT_BF16) e = launch_tc<EXT4PCF_SPLIT_BF16>(a, tm, smem, sms, s);
  else if (precision == EXT4PCF_TF32) e = launch_tc<EXT4PCF_TF32>(a, tm, smem, sms, s);
  else e = launch_tc<EXT4PCF_3XTF32>(a, tm, smem, sms, s);
  ++g_launches;
  return e;
}

// kKR expanded per component, in the layout of ext4pcf_nth_order_factors at order 4 (row mu;
// row 8 the normalisation): sign, centre code, then per bin (array, conj, coefficient of n2,
// coefficient of n3, constant); the column factor A reads s = n2 + n3.
int contraction_table_tc(int* out) {
  for (int i = 0; i < 9 * 17; ++i) out[i] = 0;
  for (int t = 0; t < kKRTypes; ++t) {
    const KRType& k = kKRHost[t];
    for (int j = 0; j < k.nmu; ++j) {
      int* r = out + k.mu[j] * 17;
      r[0] = 1;
      r[1] = k.xconj;
      const KF f[3] = {k.A[j], k.B, k.C};
      for (int l = 0; l < 3; ++l) {
        int* q = r + 2 + 5 * l;
        q[0] = f[l].arr;
        q[1] = f[l].conj;
        q[2] = (l == 0 || l == 1) ? f[l].sgn : 0;
        q[3] = (l == 0 || l == 2) ? f[l].sgn : 0;
        q[4] = f[l].off;
      }
    }
  }
  return 9 * 17;
}

}  // namespace ext4pcf

