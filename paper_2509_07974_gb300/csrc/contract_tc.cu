// Tensor-core contraction of a wave (tcgen05, sm_103a).
//
// For fixed s = n2 + n3 every natural component factorises as
//   Upsilon_mu[n2,n3](Th1,Th2,Th3) = sum_i A_i^mu[s](Th1) * KR_i[n2,n3](Th2,Th3),
//   KR_i = xt_i * B_i[n2](Th2) * C_i[n3](Th3)   (a Khatri-Rao product over the centre i),
// i.e. a complex GEMM over the centre index.  Components that share KR (mu = 0 and 2;
// mu = 1 and 5) share the GEMM.  Mapping onto tcgen05.mma (M = 128, K along centres):
//   * A operand (TMEM): 128 KR rows (n2, Th2, Th3) of one s.  Row r of the tile is TMEM
//     lane r; centre i occupies K elements (2i, 2i+1) = (re, im).  Sixteen producer warps
//     form KR on the CUDA cores and write it with tcgen05.st (warp w owns lanes
//     32 (w % 4) ..; the four warps of a lane group split the 32 centres of a stage).
//     Each stage's record slices (x~ B rows, C rows, A rows) are staged in shared memory
//     with cp.async two stages ahead.
//   * B operand (shared memory, K-major, 128-byte swizzle): column (mu, Th1, re|im) holds
//     the real embedding of A_i^mu(Th1): K rows (2i, 2i+1) = (Ar, -Ai) for the real output
//     and (Ai, Ar) for the imaginary output, so that D = A_op B_op is the complex product.
//   * D (TMEM, FP32): 128 rows x (2 * #mu * nb, padded to 16) columns.  Every 64 centres the
//     partial sum is promoted out of TMEM into FP32 registers (two D buffers alternate, so
//     the MMAs run on meanwhile); the long FP32 accumulation inside the tensor core would
//     otherwise lose bits.  The epilogue adds the sums into the FP64 output.
// Precision: BF16x3 splits every operand into bf16 hi + lo and accumulates
// hi*hi + hi*lo + lo*hi (kind::f16); 3xTF32 does the same with tf32 hi + lo (kind::tf32,
// ~22 mantissa bits per operand); TF32 uses one kind::tf32 pass.
// x~ B is formed for the whole wave by xb_kernel before the contraction.
// Pipeline: 4 (3 for 3xTF32) stages of 32 centres; full/empty mbarriers between the producers and the one
// thread that issues the MMAs; tcgen05.commit releases a stage.  Every wait is bounded by
// a clock budget; on expiry the kernel records an error code and runs to its end.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace ext4pcf {

namespace {

constexpr int kStageCentres = 32;
constexpr int kProducerWarps = 16;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 32;
constexpr uint32_t kTmemCols = 512;
constexpr int kDCols = 128;          // D region: two 64-column buffers
constexpr int kMaxNpad = 64;         // B columns: 2 * #mu * nb padded to 16 (nb <= 16)

struct KF {
  signed char arr, sgn, off, conj;  // arr 0: G, 1: W; index n = sgn * var + off
};
struct KRType {
  signed char xconj;  // 0: x, 1: x^*, 2: w
  KF B, C;            // row factors B(Th2; n2), C(Th3; n3)
  signed char nmu;
  signed char mu[2];
  KF A[2];            // column factors A(Th1; s)
};

// Khatri-Rao row types and the components that use them
#define EXT4PCF_KR_TABLE                                                                                  \
  {                                                                                                     \
    {0, {0, -1, -2, 0}, {0, -1, -3, 0}, 2, {0, 2}, {{0, 1, -3, 0}, {0, -1, -1, 1}}},                    \
    {0, {0, 1, -2, 1}, {0, -1, -3, 0}, 1, {3, 0}, {{0, 1, -3, 0}, {0, 0, 0, 0}}},                       \
    {0, {0, -1, -2, 0}, {0, 1, -1, 1}, 1, {4, 0}, {{0, 1, -3, 0}, {0, 0, 0, 0}}},                       \
    {1, {0, -1, -2, 0}, {0, -1, -1, 0}, 2, {1, 5}, {{0, 1, -1, 0}, {0, -1, -3, 1}}},                    \
    {1, {0, 1, -2, 1}, {0, -1, -1, 0}, 1, {6, 0}, {{0, 1, -1, 0}, {0, 0, 0, 0}}},                       \
    {1, {0, -1, -2, 0}, {0, 1, -3, 1}, 1, {7, 0}, {{0, 1, -1, 0}, {0, 0, 0, 0}}},                       \
    {2, {1, -1, 0, 0}, {1, -1, 0, 0}, 1, {8, 0}, {{1, 1, 0, 0}, {0, 0, 0, 0}}},                         \
  }
__constant__ KRType kKR[7] = EXT4PCF_KR_TABLE;
// host copy of the same initializer (inspection through ext4pcf_contraction_tables)
const KRType kKRHost[7] = EXT4PCF_KR_TABLE;
constexpr int kKRTypes = 7;

struct TcArgs {
  Layout L;
  const float2* rec;
  const float2* xw;
  int T;
  double* ups;
  const int4* items;  // (type, s, row0, nrows)
  int n_items;
  long long timeout;
  int* status;
};

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

// One staged block of a per-centre record: `len` consecutive complex values starting at
// record element `rec_off`; `lo` is the first multipole index (n for G, m = |n| for W).
struct Blk {
  int rec_off, len, lo, is_w;
};

__device__ __forceinline__ Blk make_blk(const Layout& L, KF f, int va, int vb) {
  int nlo = f.sgn > 0 ? va + f.off : -vb + f.off;
  int nhi = f.sgn > 0 ? vb + f.off : -va + f.off;
  Blk b;
  b.is_w = f.arr;
  if (f.arr == 0) {
    b.lo = nlo;
    b.rec_off = L.G(nlo, 0);
    b.len = (nhi - nlo + 1) * L.nb;
  } else {
    int mlo, mhi;
    if (nlo >= 0) { mlo = nlo; mhi = nhi; }
    else if (nhi <= 0) { mlo = -nhi; mhi = -nlo; }
    else { mlo = 0; mhi = max(-nlo, nhi); }
    b.lo = mlo;
    b.rec_off = L.W(mlo, 0);
    b.len = (mhi - mlo + 1) * L.nb;
  }
  return b;
}
// staged index (within the block) and conjugation of factor f at variable v, bin b
__device__ __forceinline__ int blk_index(const Blk& k, KF f, int v, int b, int nb, bool& cj) {
  const int n = f.sgn * v + f.off;
  cj = f.conj != 0;
  if (!k.is_w) return (n - k.lo) * nb + b;
  cj ^= (n < 0);
  return ((n < 0 ? -n : n) - k.lo) * nb + b;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory"); }
// the four producer warps of one centre quarter (barriers 2..5): within a stage a quarter
// reads only the staged slices that its own warps copied
__device__ __forceinline__ void quarter_sync(int q) { asm volatile("bar.sync %0, 128;" ::"r"(2 + q) : "memory"); }

// x~ times the row factor B, per centre: [5][2N+1][nb] complex, indexed by n2:
//   0: x G[-n2-2]   1: x G[n2-2]^*   2: x^* G[-n2-2]   3: x^* G[n2-2]^*   4: w W[-n2]
constexpr int kXBTypes = 5;
__constant__ signed char kXBOfType[7] = {0, 1, 0, 2, 3, 2, 4};

__global__ void xb_kernel(const Layout L, const float2* __restrict__ rec, const float2* __restrict__ xw, int T,
                          float2* __restrict__ xb) {
  const int nb = L.nb, N = L.N, nn = 2 * N + 1;
  const int per = kXBTypes * nn * nb;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < (size_t)T * per;
       k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / per), r = (int)(k % per);
    const int t = r / (nn * nb), n2 = (r / nb) % nn - N, b = r % nb;
    const float2* rc = rec + (size_t)c * L.rec;
    float2 x = xw[2 * (size_t)c], f;
    if (t == 4) {
      const int m = -n2;
      f = rc[L.W(m >= 0 ? m : -m, b)];
      if (m < 0) f.y = -f.y;
      x = xw[2 * (size_t)c + 1];
    } else {
      f = (t & 1) ? rc[L.G(n2 - 2, b)] : rc[L.G(-n2 - 2, b)];
      if (t & 1) f.y = -f.y;
      if (t >= 2) x.y = -x.y;
    }
    xb[k] = make_float2(x.x * f.x - x.y * f.y, x.x * f.y + x.y * f.x);
  }
}

constexpr int kStageBufs = 3;  // staging ring: stage k + 2 is fetched while k is formed
// A staged stage is [slot][centre]: slot e of the 32 centres is one row of kCS complex values
// (32 + 2 padding, so that rows start 4 banks apart and eight lanes reading eight slots of
// the same centres hit different banks).  A thread's eight centres are contiguous: it reads
// them with four 16-byte loads at fixed offsets.
constexpr int kCS = 34;
// staged slots per centre: a zero, the x~B and C blocks of at most the tile's n2 values
// (128 rows = 128 / nb^2 values of n2, +2 for misalignment, at most 2N+1) and two A rows
__host__ __device__ inline int stage_values(int nb, int N) {
  int rows = 128 / (nb * nb) + 2;
  if (rows > 2 * N + 1) rows = 2 * N + 1;
  return (1 + 2 * rows * nb + 2 * nb) | 1;
}
// stages per TMEM partial sum (64 centres): the tensor core's FP32 accumulation loses bits
// in proportion to the MMAs it accumulates (measured: ~3e-4 over 750 MMAs, ~5e-5 over
// 96, ~1.5e-4 over 192 for 3xTF32), so partial sums are short and summed in registers
constexpr int kPromote = 2;
constexpr int kDBuf = 64;    // two D buffers of 64 columns (npad <= 64)
constexpr int kQuarter = kStageCentres / (kProducerWarps / 4);  // centres per producer warp

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

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
contract_tc_kernel(const TcArgs args, const float2* __restrict__ xbarr) {
  using P = TcPrec<PREC>;
  constexpr int kSt = P::kStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const Layout L = args.L;
  const int nb = L.nb, N = L.N, nn = 2 * N + 1, nb2 = nb * nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int tile_bytes = kMaxNpad * 128;  // one 128-byte-wide K-atom (npad <= 64)
  constexpr int stage_bytes = P::kAtoms * tile_bytes;
  const int sc_max = stage_values(nb, N);
  float2* stg = reinterpret_cast<float2*>(sm + kSt * stage_bytes);
  int* gmap = reinterpret_cast<int*>(stg + kStageBufs * sc_max * kCS);  // [sc_max]
  uint64_t* full = reinterpret_cast<uint64_t*>(gmap + ((sc_max + 1) & ~1));
  uint64_t* empty = full + kSt;
  uint64_t* dfull = empty + kSt;  // [2]: a D buffer holds a finished partial sum
  uint64_t* dempty = dfull + 2;   // [2]: the producers have read it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dempty + 2);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int k = 0; k < kSt; ++k) {
      mbar_init(&full[k], kProducers);
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&dfull[k], 1);
      mbar_init(&dempty[k], kProducers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long budget = args.timeout;
  const int nstage = (args.T + kStageCentres - 1) / kStageCentres;
  const int nsub = (nstage + kPromote - 1) / kPromote;
  const size_t xb_stride = (size_t)kXBTypes * nn * nb;
  int err = 0;

  long long gk = 0;  // stages handled by this CTA (phases of full / empty)
  long long gs = 0;  // partial sums handled by this CTA (phases of dfull / dempty)
  for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
    const int4 item = args.items[it];
    const int type = item.x, s = item.y, row0 = item.z, nrows = item.w;
    const KRType kr = kKR[type];
    const int nmu = kr.nmu;
    const int ncols = 2 * nmu * nb;
    const int npad = (ncols + 15) / 16 * 16;
    const int n2a = max(-N, s - N);
    // the tile's rows span n2 in [t2a, t2b]; staged per centre: [0] zero, x~B rows
    // [t2a, t2b], C rows for n3 = s - n2, A_0(s), A_1(s)
    const int t2a = n2a + row0 / nb2, t2b = n2a + (row0 + nrows - 1) / nb2;
    const int xb_len = (t2b - t2a + 1) * nb;
    const int xb_off = (kXBOfType[type] * nn + (t2a + N)) * nb;
    const Blk bkC = make_blk(L, kr.C, s - t2b, s - t2a);
    const Blk bkA0 = make_blk(L, kr.A[0], s, s);
    const Blk bkA1 = nmu > 1 ? make_blk(L, kr.A[1], s, s) : Blk{0, 0, 0, 0};
    const int bC = 1 + xb_len, bA0 = bC + bkC.len, bA1 = bA0 + bkA0.len;
    const int sc = (bA1 + bkA1.len) | 1;
    if (warp < kProducerWarps) {
      // ------------------------------------------------------------------ producers
      // record offsets of the staged values after the x~B block (-1: nothing to copy)
      for (int e = bC + tid; e < sc; e += kProducers) {
        int m = -1;
        if (e < bA0) m = bkC.rec_off + (e - bC);
        else if (e < bA1) m = bkA0.rec_off + (e - bA0);
        else if (e < bA1 + bkA1.len) m = bkA1.rec_off + (e - bA1);
        gmap[e] = m;
      }
      producers_sync();
      const int grp = warp & 3, quarter = warp >> 2;
      const int rl = grp * 32 + lane;  // tile row = TMEM lane
      const bool row_ok = rl < nrows;
      const int rr = row0 + (row_ok ? rl : 0);
      const int n2 = n2a + rr / nb2, b2 = (rr / nb) % nb, b3 = rr % nb, n3 = s - n2;
      bool cjC;
      int iB = 1 + (n2 - t2a) * nb + b2;
      int iC = bC + blk_index(bkC, kr.C, n3, b3, nb, cjC);
      const float sgnC = cjC ? -1.f : 1.f;
      if (!row_ok) { iB = 0; iC = 0; }
      // B-operand words of this thread: the quarter's 128 threads write the tile's K range of
      // its eight centres; column bn, centres 8 quarter + cpt bq + j (j < cpt)
      const int tq = tid & 127;
      const int cpt = npad <= 16 ? 1 : (npad <= 32 ? 2 : 4);
      const int tpc = 8 / cpt;
      const int bn = tq / tpc, bq = tq % tpc;
      const int cb0 = quarter * kQuarter + bq * cpt;
      uint32_t boff[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        boff[j] = PREC == EXT4PCF_SPLIT_BF16 ? sw128_word_off(bn, cb0 + j, kMaxNpad)
                                             : sw128_word_off(bn, 2 * (cb0 + j), kMaxNpad);
      int iA = 0, bo = 0;
      float sgnA = 1.f;
      if (bn < ncols) {
        const int g = bn / (2 * nb), b1 = (bn >> 1) % nb;
        bool cjA;
        bo = bn & 1;
        iA = (g ? bA1 : bA0) + blk_index(g ? bkA1 : bkA0, kr.A[g], s, b1, nb, cjA);
        sgnA = cjA ? -1.f : 1.f;
      }
      // copy plan of this thread for every stage (16 threads per centre): staged slots
      // e = 1 + sub + 16 j; slots j < jx come from the x~B array (source offset e - 1 from
      // the item's x~B row block), slots jx <= j < jr from the record (offset coff[j])
      constexpr int kMaxCopies = 12;  // 16 * 12 >= stage_values(nb, N) for every supported shape
      // record offsets (< 2^16 for every supported shape: at most (14 * 40 + 13) * 32
      // elements per record), two per register
      uint32_t coff2[kMaxCopies / 2];
      const int sub = tid & 15;
      const int e_end = bA1 + bkA1.len;  // slots past the A blocks are padding
      const int jx = max(0, (bC - 1 - sub + 15) / 16), jr = max(0, (e_end - 1 - sub + 15) / 16);
#pragma unroll
      for (int j = 0; j < kMaxCopies; j += 2) {
        const int e0 = 1 + sub + 16 * j, e1 = e0 + 16;
        const uint32_t o0 = (e0 >= bC && e0 < e_end) ? (uint32_t)gmap[e0] : 0u;
        const uint32_t o1 = (e1 >= bC && e1 < e_end) ? (uint32_t)gmap[e1] : 0u;
        coff2[j / 2] = o0 | (o1 << 16);
      }
      // source pointers of the next stage to fetch (advanced by 32 centres per stage)
      const int ci0 = tid >> 4;
      const float2* xs_next = xbarr + (size_t)ci0 * xb_stride + xb_off + sub;
      const float2* rc_next = args.rec + (size_t)ci0 * L.rec;
      const size_t xs_step = (size_t)kStageCentres * xb_stride, rc_step = (size_t)kStageCentres * L.rec;
      int fetch_buf = 0;  // staging buffer of the next stage to fetch
      // copy one stage's slices (stages are fetched in order); tails are zero-filled
      auto issue = [&](int k) {
        if (k < nstage) {
          float2* d = stg + (size_t)fetch_buf * sc_max * kCS + ci0;  // slot e at d[e * kCS]
          const int c = k * kStageCentres + ci0;
          if (c < args.T) {
            if (sub == 0) d[0] = make_float2(0.f, 0.f);
            float2* dd = d + (1 + sub) * kCS;
#pragma unroll
            for (int j = 0; j < kMaxCopies; ++j) {
              if (j >= jr) break;
              if (j < jx) cp_async8(dd + 16 * kCS * j, xs_next + 16 * j);
              else cp_async8(dd + 16 * kCS * j, rc_next + ((coff2[j / 2] >> (16 * (j & 1))) & 0xFFFFu));
            }
          } else {
            for (int e = sub; e < sc; e += 16) d[e * kCS] = make_float2(0.f, 0.f);
          }
          xs_next += xs_step;
          rc_next += rc_step;
          fetch_buf = fetch_buf == kStageBufs - 1 ? 0 : fetch_buf + 1;
        }
        cp_async_commit();
      };
      issue(0);
      issue(1);
      float accD[16];  // FP32 sums of the promoted partials: this row, 16 columns
#pragma unroll
      for (int j = 0; j < 16; ++j) accD[j] = 0.f;
      auto promote = [&](long long g) {  // read partial sum g from its D buffer
        const int buf = (int)(g & 1);
        if (!mbar_wait(&dfull[buf], (uint32_t)((g >> 1) & 1), budget)) err = 1;
        tc_fence_after();
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(grp * 32) << 16) + buf * kDBuf + quarter * 16, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) accD[j] += __uint_as_float(v[j]);
        tc_fence_before();
        mbar_arrive(&dempty[buf]);
      };
      const long long gs0 = gs;
      int slot = (int)(gk % kSt);
      uint32_t ph = (uint32_t)((gk / kSt) & 1);
      int read_buf = 0;
      for (int k = 0; k < nstage; ++k, ++gk) {
        cp_async_wait<1>();
        quarter_sync(quarter);
        issue(k + 2);
        const float2* st = stg + (size_t)read_buf * sc_max * kCS;
        read_buf = read_buf == kStageBufs - 1 ? 0 : read_buf + 1;
        if (!mbar_wait(&empty[slot], ph ^ 1u, budget)) err = 1;
        tc_fence_after();
        // B operand (shared memory, swizzled): real embedding of A(Th1) for 4 centres
        unsigned char* bt = sm + slot * stage_bytes;
        if (bn < npad) {
          const float2* ap = st + iA * kCS + cb0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (j >= cpt) break;
            float2 a = ap[j];
            a.y *= sgnA;
            const float v0 = bo ? a.y : a.x;
            const float v1 = bo ? a.x : -a.y;
            if (PREC == EXT4PCF_SPLIT_BF16) {
              uint32_t h, l;
              split_bf16(v0, v1, h, l);
              *reinterpret_cast<uint32_t*>(bt + boff[j]) = h;
              *reinterpret_cast<uint32_t*>(bt + tile_bytes + boff[j]) = l;
            } else if (PREC == EXT4PCF_TF32) {
              *reinterpret_cast<float2*>(bt + boff[j]) = make_float2(v0, v1);
            } else {
              uint32_t h0, l0, h1, l1;
              split_tf32(v0, h0, l0);
              split_tf32(v1, h1, l1);
              *reinterpret_cast<uint2*>(bt + boff[j]) = make_uint2(h0, h1);
              *reinterpret_cast<uint2*>(bt + 2 * tile_bytes + boff[j]) = make_uint2(l0, l1);
            }
          }
        }
        // A operand (TMEM): this row's Khatri-Rao values x~B * C for 8 centres
        // x~B and C of this row for the quarter's eight centres (contiguous in the slot rows)
        float2 xbv[kQuarter], cvv[kQuarter];
        {
          const float4* b4 = reinterpret_cast<const float4*>(st + iB * kCS + quarter * kQuarter);
          const float4* c4 = reinterpret_cast<const float4*>(st + iC * kCS + quarter * kQuarter);
#pragma unroll
          for (int q = 0; q < kQuarter / 2; ++q) {
            const float4 tb = b4[q], tc = c4[q];
            xbv[2 * q] = make_float2(tb.x, tb.y);
            xbv[2 * q + 1] = make_float2(tb.z, tb.w);
            cvv[2 * q] = make_float2(tc.x, tc.y);
            cvv[2 * q + 1] = make_float2(tc.z, tc.w);
          }
        }
        const uint32_t acol = tmem + ((uint32_t)(grp * 32) << 16) + kDCols + slot * P::kStageCols;
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
        fence_async_smem();
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&full[slot]);
        if (++slot == kSt) { slot = 0; ph ^= 1u; }
        // a partial sum finished one promotion block ago is read while the MMAs run on
        if ((k % kPromote) == kPromote - 1 && k / kPromote >= 1) promote(gs0 + k / kPromote - 1);
      }
      cp_async_wait<0>();
      // the remaining partial sums of this item: the loop read partials 0 .. F-2
      // (F = complete promotion blocks)
      const int read_in_loop = max(0, nstage / kPromote - 1);
      for (long long g = gs0 + read_in_loop; g < gs0 + nsub; ++g) promote(g);
      gs = gs0 + nsub;
      // ------------------------------------------------------------------ epilogue
      if (row_ok) {
        const size_t nb3 = (size_t)nb2 * nb;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int n = quarter * 16 + j;
          if (n < ncols) {
            const int g = n / (2 * nb), b1 = (n >> 1) % nb;
            const int mu = kr.mu[g];
            const size_t o = ((((size_t)mu * nn + (n2 + N)) * nn + (n3 + N)) * nb3) + (size_t)b1 * nb2 +
                             (size_t)b2 * nb + b3;
            double* p = args.ups + 2 * o;
            p[0] += (double)accD[j];
            p[1] += (double)accD[j + 1];
          }
        }
      }
      producers_sync();
    } else {
      // ------------------------------------------------------------------ MMA issuer
      if (lane == 0) {
        const uint32_t id = PREC == EXT4PCF_SPLIT_BF16 ? idesc(1u, npad) : idesc(2u, npad);
        int slot = (int)(gk % kSt);
        uint32_t ph = (uint32_t)((gk / kSt) & 1);
        for (int k = 0; k < nstage; ++k, ++gk) {
          const long long g = gs + k / kPromote;
          const int buf = (int)(g & 1);
          const bool first = (k % kPromote) == 0;
          if (first && g >= 2) {
            if (!mbar_wait(&dempty[buf], (uint32_t)(((g >> 1) - 1) & 1), budget)) err = 1;
          }
          if (!mbar_wait(&full[slot], ph, budget)) err = 1;
          tc_fence_after();
          const uint32_t d = tmem + buf * kDBuf;
          const uint32_t a0 = tmem + kDCols + slot * P::kStageCols;
          const uint32_t b0 = saddr(sm + slot * stage_bytes);
          if (PREC == EXT4PCF_SPLIT_BF16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // K = 16 bf16 = 8 centres per MMA
              const uint64_t bh = desc_sw128(b0 + q * 32), bl = desc_sw128(b0 + tile_bytes + q * 32);
              mma_f16(d, a0 + q * 8, bh, id, (!first || q > 0) ? 1u : 0u);
              mma_f16(d, a0 + q * 8, bl, id, 1u);
              mma_f16(d, a0 + 32 + q * 8, bh, id, 1u);
            }
          } else if (PREC == EXT4PCF_TF32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // K = 8 fp32 = 4 centres per MMA
              const uint64_t b = desc_sw128(b0 + (q >> 2) * tile_bytes + (q & 3) * 32);
              mma_tf32(d, a0 + q * 8, b, id, (!first || q > 0) ? 1u : 0u);
            }
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // hi*hi + hi*lo + lo*hi, K = 8 fp32 per MMA
              const uint32_t bo_ = (q >> 2) * tile_bytes + (q & 3) * 32;
              const uint64_t bh = desc_sw128(b0 + bo_), bl = desc_sw128(b0 + 2 * tile_bytes + bo_);
              mma_tf32(d, a0 + q * 8, bh, id, (!first || q > 0) ? 1u : 0u);
              mma_tf32(d, a0 + q * 8, bl, id, 1u);
              mma_tf32(d, a0 + 64 + q * 8, bh, id, 1u);
            }
          }
          mma_commit(&empty[slot]);
          if ((k % kPromote) == kPromote - 1 || k == nstage - 1) mma_commit(&dfull[buf]);
          if (++slot == kSt) { slot = 0; ph ^= 1u; }
        }
      } else {
        gk += nstage;
      }
      gs += nsub;
      __syncwarp();
    }
  }
  // drain: the last partial sum was read by the producers, so no MMA is in flight
  if (err) atomicExch(args.status, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

size_t tc_smem_bytes(int nb, int N, int prec) {
  const bool x3 = prec == EXT4PCF_3XTF32;
  const int st = x3 ? TcPrec<EXT4PCF_3XTF32>::kStages : 4;
  const int atoms = x3 ? TcPrec<EXT4PCF_3XTF32>::kAtoms : 2;
  const int sc = stage_values(nb, N);
  return (size_t)st * atoms * kMaxNpad * 128 + (size_t)kStageBufs * sc * kCS * 8 +
         (size_t)((sc + 1) & ~1) * 4 + 1024 + 256;
}

template <int PREC>
cudaError_t launch_tc(const TcArgs& a, const float2* xb, size_t smem, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contract_tc_kernel<PREC><<<sms, kThreads, smem, s>>>(a, xb);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Layout& L, int precision) {
  if (precision != EXT4PCF_SPLIT_BF16 && precision != EXT4PCF_TF32 && precision != EXT4PCF_3XTF32) return false;
  return L.nb >= 1 && 4 * L.nb <= kMaxNpad && tc_smem_bytes(L.nb, L.N, precision) <= 227 * 1024;
}

void tc_build_items(const Layout& L, std::vector<int4>& items) {
  items.clear();
  const int N = L.N, nb2 = L.nb * L.nb;
  for (int t = 0; t < kKRTypes; ++t)
    for (int s = -2 * N; s <= 2 * N; ++s) {
      const int lo = s - N > -N ? s - N : -N, hi = s + N < N ? s + N : N;
      const int rows = (hi - lo + 1) * nb2;
      for (int r0 = 0; r0 < rows; r0 += 128) items.push_back(make_int4(t, s, r0, rows - r0 < 128 ? rows - r0 : 128));
    }
}

size_t contract_tc_xb_bytes(const Layout& L, int T) {
  return (size_t)T * kXBTypes * (2 * L.N + 1) * L.nb * sizeof(float2);
}

cudaError_t contract_wave_tc(const Layout& L, const float2* rec, const float2* xw, int T, double* ups,
                             int precision, const int4* items, int n_items, float2* xb, int* status,
                             long long timeout, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  {
    const size_t total = (size_t)T * kXBTypes * (2 * L.N + 1) * L.nb;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 65536);
    xb_kernel<<<blocks, 256, 0, s>>>(L, rec, xw, T, xb);
    ++g_launches;
  }
  TcArgs a;
  a.L = L; a.rec = rec; a.xw = xw; a.T = T; a.ups = ups;
  a.items = items; a.n_items = n_items;
  a.timeout = timeout; a.status = status;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = tc_smem_bytes(L.nb, L.N, precision);
  cudaError_t e;
  if (precision == EXT4PCF_SPLIT_BF16) e = launch_tc<EXT4PCF_SPLIT_BF16>(a, xb, smem, sms, s);
  else if (precision == EXT4PCF_TF32) e = launch_tc<EXT4PCF_TF32>(a, xb, smem, sms, s);
  else e = launch_tc<EXT4PCF_3XTF32>(a, xb, smem, sms, s);
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

