// Split-FP16 tensor-core contraction of a wave (tcgen05 kind::f16, sm_103a).
//
// The GEMM is that of the other tensor-core forms (contract_tc.cu): for fixed s = n2 + n3 the
// Khatri-Rao rows x~B[n2](Th2) C[n3](Th3) over the bin pairs Th2 <= Th3 are multiplied with the
// column factors A^mu[s](Th1), K running over the centres, and the sums go to the reduced array
// of the Theta2 <-> Theta3 symmetry (Table tab:4PCFSymm).  This kernel arranges the data so
// that forming the rows on the CUDA cores -- the part that bounds the other forms -- takes
// about as long as the tensor core's three passes:
//  * Power-of-two row scales.  A pre-pass finds the largest |component| of every row of the
//    wave array (x~B, G, W rows) and the transpose writes each row times 2^k, its largest
//    component in [2^6, 2^7).  A product of two rows is then below 2^15, inside the fp16
//    range, with no per-value scaling in the kernel; the epilogue takes out the exact factor
//    2^-(k_B + k_C + k_A).
//  * Planar staging.  Per 16 centres a row holds their 16 real parts, then their 16 imaginary
//    parts (128 bytes), so that two centres' real (or imaginary) parts form one 64-bit register
//    pair and the complex products run on the packed f32x2 pipe.
//  * Stage-major wave array.  The array is laid out [stage of 64 centres][row][512 bytes], the
//    16-byte chunks of every 128-byte quarter XOR-permuted by the row index mod 8 (the 128-byte
//    swizzle, applied by the transpose).  The rows a work item needs for one stage (its x~B,
//    C and A blocks) are then four contiguous ranges, fetched with four plain bulk copies
//    (cp.async.bulk) instead of one tensor box per 8 rows and 16 centres: the copy engine's
//    per-request cost, not bandwidth, bounded the boxed staging.  Eight lanes reading eight
//    consecutive rows at the same logical chunk hit eight different bank groups.
//  * K order.  In every group of 8 centres (one MMA, K = 16 halves) K = 0..7 holds the real
//    and K = 8..15 the imaginary parts of the row values; the column operand holds (A_r, -A_i)
//    for the real and (A_i, A_r) for the imaginary output at the same K.
//  * W for both signs of m.  W_{-m} = conj W_m is written out, so the conjugation of every
//    factor is fixed by the row type and uniform over a work item.
//  * 64-centre stages and ring counters without divisions: each producer thread forms 16
//    values of its row per stage between two barrier crossings.
// Precision: every operand is split into fp16 hi + lo (22 significant bits) and the MMAs
// accumulate hi*hi + hi*lo + lo*hi in FP32 over one stage; the stage's partial sums are
// promoted into FP32 registers while the next stage runs, and the epilogue adds them into the
// FP64 reduced array.
// Every wait is bounded by a clock budget; on expiry the kernel records an error code, runs to
// its end, waits for its own MMAs and copies and frees its TMEM.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kr_table.cuh"
#include "tc_ptx.cuh"

namespace ext4pcf {

namespace {

constexpr int kHCentres = 64;                        // centres per stage
constexpr int kHProducerWarps = 16;
constexpr int kHThreads = kHProducerWarps * 32 + 64; // + the MMA issuer and the TMA loader warp
constexpr int kHWarpMma = kHProducerWarps, kHWarpLoad = kHProducerWarps + 1;
constexpr int kHSlots = 3;                           // A (TMEM) and B (shared) ring depth
constexpr int kHACols = 128;                         // TMEM columns per A slot: 64 hi + 64 lo
constexpr int kHDCols = 128;                         // two D buffers of 64 columns
constexpr int kHMaxIn = 4;                           // staged-input ring depth at most
constexpr uint32_t kHTmemCols = 512;
constexpr int kHScaleTop = 6;                        // rows scaled into [2^6, 2^7)

// exponent k of the row scale 2^k for a row whose largest |component| has the float bits m
__host__ __device__ __forceinline__ int h_scale_exp(unsigned mbits) {
#ifdef __CUDA_ARCH__
  const float m = __uint_as_float(mbits);
  if (!(m > 0.f)) return 0;
  const int k = kHScaleTop - ilogbf(m);
  return k < -100 ? -100 : (k > 100 ? 100 : k);
#else
  (void)mbits;
  return 0;
#endif
}
__device__ __forceinline__ float h_pow2f(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ double h_pow2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Row of the transposed wave array at one centre (rc: the centre's record, x = w gamma, w):
//   rows [0, row_g)      x~B per x~B type: (type, n2 + N + 1, bin), n2 in [-N-1, N+1]
//   rows [row_g, row_w)  G_n(bin), n in [-2N-3, 2N-1]
//   rows [row_w, rows)   W_m(bin), m in [-2N, 2N]
__device__ __forceinline__ float2 hwave_value(const Layout& L, const float2* __restrict__ rc, float2 x, float w,
                                              int r, int row_g, int row_w) {
  const int nb = L.nb, N = L.N, nx = 2 * N + 3;
  if (r >= row_w) {
    const int m = (r - row_w) / nb - 2 * N, b = (r - row_w) % nb;
    float2 f = rc[L.W(m >= 0 ? m : -m, b)];
    if (m < 0) f.y = -f.y;
    return f;
  }
  if (r >= row_g) return rc[L.oG + (r - row_g)];
  const int t = r / (nx * nb), n2 = (r / nb) % nx - N - 1, b = r % nb;
  float2 f;
  if (t == 4) {
    const int m = -n2;  // w W[-n2], |n2| <= N
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

// largest |component| of every row over the wave's centres: 32 rows x 128 centres per block
// (records of the wave's live centres only: padding records are never read)
__global__ void __launch_bounds__(256) hwave_rowmax_kernel(const Layout L, const float2* __restrict__ rec,
                                                           const float2* __restrict__ xw, const WavePlan plan,
                                                           int row_g, int row_w, int rows,
                                                           unsigned* __restrict__ rowmax) {
  __shared__ float part[8][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 128;
  if (c0 >= plan.total) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, r = r0 + tx;
  float m = 0.f;
  if (r < rows) {
    for (int k = 0; k < 16; ++k) {
      const int c = c0 + ty + 8 * k;
      int j = 0;
      const int si = c < plan.total ? seg_of(plan, c, &j) : -1;
      if (si >= 0 && j < seg_live(plan.seg[si])) {
        const float2 v = hwave_value(L, rec + (size_t)c * L.rec, xw[2 * (size_t)c], xw[2 * (size_t)c + 1].x, r,
                                     row_g, row_w);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
  }
  part[ty][tx] = m;
  __syncthreads();
  if (ty == 0 && r < rows) {
    for (int k = 1; k < 8; ++k) m = fmaxf(m, part[k][tx]);
    if (m > 0.f) atomicMax(&rowmax[r], __float_as_uint(m));  // non-negative floats order as integers
  }
}

// The transposed, scaled, planar wave array, stage-major: record c of row r sits in stage
// c / 64 at float (c / 64 * rows + r) * 128 + q * 32 + ((k ^ (r % 8)) * 4) + c % 4, with
// q = (c % 64) / 16 the quarter and k = (c % 16) / 4 (real part) or 4 + (c % 16) / 4
// (imaginary part) the logical 16-byte chunk.
// Padding records (between segments, past a segment's live centres, past the wave up to a
// multiple of 64) are written as zeros.
__global__ void __launch_bounds__(256) hwave_transpose_kernel(const Layout L, const float2* __restrict__ rec,
                                                              const float2* __restrict__ xw, const WavePlan plan,
                                                              int row_g, int row_w, int rows,
                                                              const unsigned* __restrict__ rowmax,
                                                              float* __restrict__ out) {
  __shared__ float2 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int Tp = (plan.total + kHCentres - 1) / kHCentres * kHCentres;
  if (c0 >= Tp) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + ty + 8 * k, r = r0 + tx;
    float2 v = make_float2(0.f, 0.f);
    int j = 0;
    const int si = c < plan.total ? seg_of(plan, c, &j) : -1;
    if (si >= 0 && j < seg_live(plan.seg[si]) && r < rows)
      v = hwave_value(L, rec + (size_t)c * L.rec, xw[2 * (size_t)c], xw[2 * (size_t)c + 1].x, r, row_g, row_w);
    tile[ty + 8 * k][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    if (r < rows) {
      const float sc = h_pow2f(h_scale_exp(rowmax[r]));
      const float2 v = tile[tx][ty + 8 * k];
      const int q = (c & 63) >> 4, kre = (c & 15) >> 2, sw = r & 7;
      float* o = out + ((size_t)(c >> 6) * rows + r) * 128 + q * 32 + (c & 3);
      o[(kre ^ sw) * 4] = v.x * sc;
      o[((4 + kre) ^ sw) * 4] = v.y * sc;
    }
  }
}

struct HArgs {
  Layout L;
  WavePlan plan;      // the wave's segments (a segment starts at a stage boundary)
  double* red;        // reduced outputs [slot][9][2N+3][2N+3][nb][npairs] (complex, FP64)
  size_t red_stride;  // doubles per slot
  int npairs;
  const int4* items;  // (type, s, row0, nrows | (n2 of row 0 of the s block + 64) << 8)
  int n_items;
  int row_g, row_w;   // first G row and first W row of the wave array
  const unsigned* rowmax;  // largest |component| per row (float bits): the row scales
  const float* wave;  // the stage-major wave array
  int rows;           // its rows
  int in_stages;      // staged-input ring depth
  int stage_rows;     // rows per staged stage
  int npad_max;       // rows of a B tile: 2 * 2 * nb rounded up to 16
  long long timeout;
  int* status;
};

// rows of factor f for its variable in [va, vb]: first row in the wave array, count, and the
// multipole index of the first row
struct HBlk {
  int row0, len, lo;
};
__device__ __forceinline__ HBlk hblk(const HArgs& a, KF f, int va, int vb) {
  const int nb = a.L.nb, N = a.L.N;
  const int nlo = f.sgn > 0 ? va + f.off : -vb + f.off;
  const int nhi = f.sgn > 0 ? vb + f.off : -va + f.off;
  HBlk b;
  b.lo = nlo;
  b.len = (nhi - nlo + 1) * nb;
  b.row0 = f.arr == 0 ? a.row_g + (nlo + 2 * N + 3) * nb : a.row_w + (nlo + 2 * N) * nb;
  return b;
}
__device__ __forceinline__ int hblk_index(const HBlk& k, KF f, int v, int b, int nb) {
  return (f.sgn * v + f.off - k.lo) * nb + b;
}

// Geometry of one work item: the staged blocks (x~B rows, C rows, A rows) and their first
// rows in a staged stage (packed one after the other)
struct HGeo {
  int s, row0, nrows, n2a, t2a, t2b;
  HBlk bx, bc, ba0, ba1;
  int sx, sc, sa0, sa1;
};
__device__ __forceinline__ HGeo hgeo(const HArgs& a, int4 item, const KRType& kr) {
  const int nb = a.L.nb, N = a.L.N, nx = 2 * N + 3;
  HGeo g;
  g.s = item.y;
  g.row0 = item.z;
  g.nrows = item.w & 0xFF;
  g.n2a = (item.w >> 8) - 64;
  g.t2a = g.n2a + g.row0 / a.npairs;
  g.t2b = g.n2a + (g.row0 + g.nrows - 1) / a.npairs;
  g.bx.row0 = (kXBOfType[item.x] * nx + (g.t2a + N + 1)) * nb;
  g.bx.len = (g.t2b - g.t2a + 1) * nb;
  g.bx.lo = g.t2a;
  g.bc = hblk(a, kr.C, g.s - g.t2b, g.s - g.t2a);
  g.ba0 = hblk(a, kr.A[0], g.s, g.s);
  g.ba1 = kr.nmu > 1 ? hblk(a, kr.A[1], g.s, g.s) : HBlk{0, 0, 0};
  g.sx = 0;
  g.sc = g.bx.len;
  g.sa0 = g.sc + g.bc.len;
  g.sa1 = g.sa0 + g.ba0.len;
  return g;
}

// packed FP32x2 arithmetic on register pairs (x in the low word)
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// fp16 hi/lo split of a pair: hi = (fp16(a), fp16(b)) with a in the low half, lo the same of
// the exact residuals a - hi_a, b - hi_b (formed by one mixed-precision FMA each)
__device__ __forceinline__ void split_h2(unsigned long long v, uint32_t& hi, uint32_t& lo) {
  asm("{\n .reg .f32 a, b, r0, r1;\n .reg .b16 h0, h1, m1;\n"
      " mov.b64 {a, b}, %2;\n"
      " cvt.rn.f16x2.f32 %0, b, a;\n"
      " mov.b32 {h0, h1}, %0;\n"
      " mov.b16 m1, 0xBC00;\n"
      " fma.rn.f32.f16 r0, h0, m1, a;\n"
      " fma.rn.f32.f16 r1, h1, m1, b;\n"
      " cvt.rn.f16x2.f32 %1, r1, r0;\n}\n"
      : "=r"(hi), "=r"(lo)
      : "l"(v));
}
// 16 bytes of shared memory as two register pairs
__device__ __forceinline__ void lds_2x64(uint32_t addr, unsigned long long& a, unsigned long long& b) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr) : "memory");
}
__device__ __forceinline__ unsigned long long lds_64(uint32_t addr) {
  unsigned long long a;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(a) : "r"(addr) : "memory");
  return a;
}
__device__ __forceinline__ void sts_32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// The Khatri-Rao values of one row for 8 centres (group h of the thread's 16): x~B at PB, C at
// PC (shared addresses of the rows in the staged stage, swizzle term folded in: chunk c is at
// P ^ (c << 4)); CJ: C enters conjugated.  Writes hi / lo words 0..7: four pairs of real parts,
// then four pairs of imaginary parts.  One 16-byte chunk (four centres) at a time.
template <bool CJ>
__device__ __forceinline__ void kr_group(uint32_t PB, uint32_t PC, int h, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const uint32_t re_off = (uint32_t)(2 * h + c) << 4, im_off = (uint32_t)(4 + 2 * h + c) << 4;
    unsigned long long xr[2], xi[2], cr[2], ci[2];
    lds_2x64(PB ^ re_off, xr[0], xr[1]);
    lds_2x64(PB ^ im_off, xi[0], xi[1]);
    lds_2x64(PC ^ re_off, cr[0], cr[1]);
    lds_2x64(PC ^ im_off, ci[0], ci[1]);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      unsigned long long re, im;
      if (CJ) {  // x~B conj(C)
        re = f2fma(xi[p], ci[p], f2mul(xr[p], cr[p]));
        im = f2sub(f2mul(xi[p], cr[p]), f2mul(xr[p], ci[p]));
      } else {
        re = f2sub(f2mul(xr[p], cr[p]), f2mul(xi[p], ci[p]));
        im = f2fma(xr[p], ci[p], f2mul(xi[p], cr[p]));
      }
      split_h2(re, hi[2 * c + p], lo[2 * c + p]);
      split_h2(im, hi[4 + 2 * c + p], lo[4 + 2 * c + p]);
    }
  }
}

// Warp roles: warps 0..15 form the A operand (Khatri-Rao rows, TMEM) and the B operand
// (shared memory) of each stage; warp 16 issues the MMAs (one thread); warp 17 stages each
// stage's rows of the wave array with TMA (one thread).  Rings and their mbarriers (counts in
// brackets):
//   staged input  in_full [1 + TMA bytes] / in_empty [16 producer warps]
//   A and B       ab_full [16 producer warps] / ab_empty [1, tcgen05.commit]
//   partial sums  dfull [1, tcgen05.commit] / dempty [16 producer warps]
__global__ void __launch_bounds__(kHThreads, 1)
contract_h16_kernel(const __grid_constant__ HArgs args) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const Layout L = args.L;
  const int nb = L.nb, N = L.N, npairs = args.npairs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t atom_bytes = (uint32_t)args.npad_max * 128u;  // one 128-byte-wide K-atom of a B tile
  const uint32_t bslot_bytes = 4u * atom_bytes;                  // hi tile (2 atoms) | lo tile (2 atoms)
  const uint32_t in_bytes = (uint32_t)args.stage_rows * 512u;    // one staged stage: rows of 512 bytes
  const int S_in = args.in_stages;
  unsigned char* in_base = sm + kHSlots * bslot_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(in_base + (size_t)S_in * in_bytes);
  uint64_t* in_full = bars;
  uint64_t* in_empty = in_full + kHMaxIn;
  uint64_t* ab_full = in_empty + kHMaxIn;
  uint64_t* ab_empty = ab_full + kHSlots;
  uint64_t* dfull = ab_empty + kHSlots;  // [2]
  uint64_t* dempty = dfull + 2;          // [2]
  uint64_t* drain = dempty + 2;          // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kHTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int k = 0; k < S_in; ++k) {
      mbar_init(&in_full[k], 1);
      mbar_init(&in_empty[k], kHProducerWarps);
    }
    for (int k = 0; k < kHSlots; ++k) {
      mbar_init(&ab_full[k], kHProducerWarps);
      mbar_init(&ab_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&dfull[k], 1);
      mbar_init(&dempty[k], kHProducerWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long budget = args.timeout;
  int err = 0;
  // bounded wait on an mbarrier phase; the first wait of the CTA that runs out of its budget
  // raises the abort flag, after which every wait gives up at once
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

  if (warp < kHProducerWarps) {
    // ---------------------------------------------------------------------- producers
    const int grp = warp & 3, qq = warp >> 2;  // TMEM lane group; 16-centre quarter of a stage
    const uint32_t in_addr = saddr(in_base), b_addr = saddr(sm);
    int islot = 0, aslot = 0;
    uint32_t iph = 0, aph = 0;
    long long gs = 0;  // partial sums (stages) so far
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const int4 item = args.items[it];
      const KRType kr = kKR[item.x];
      const HGeo g = hgeo(args, item, kr);
      const int nmu = kr.nmu, ncols = 2 * nmu * nb, nv = nmu * nb;
      const int npad = (ncols + 15) & ~15;
      const int rl = grp * 32 + lane;  // tile row = TMEM lane
      const bool row_ok = rl < g.nrows;
      const int rr = g.row0 + (row_ok ? rl : 0);
      const int n2 = g.n2a + rr / npairs, n3 = g.s - n2;
      int b2, b3;
      pair_of(rr % npairs, nb, b2, b3);
      const int eB = g.sx + (n2 - g.t2a) * nb + b2;
      const int eC = g.sc + hblk_index(g.bc, kr.C, n3, b3, nb);
      const bool cjC = kr.C.conj != 0;
      // this row's x~B and C rows, quarter qq, in a staged stage, with the swizzle term of their
      // rows in the wave array folded in (chunk c at P ^ (c << 4))
      const int rB = g.bx.row0 + (eB - g.sx), rC = g.bc.row0 + (eC - g.sc);
      const uint32_t xB0 = (uint32_t)eB * 512u + qq * 128u + ((uint32_t)(rB & 7) << 4);
      const uint32_t xC0 = (uint32_t)eC * 512u + qq * 128u + ((uint32_t)(rC & 7) << 4);
      // the B columns this warp forms: column pairs v = warp, warp + 16 (component slot v / nb,
      // Th1 = v % nb); lane = centres 2 lane, 2 lane + 1 of the stage
      // shared offsets: aoff = the lane's two real parts of A (the imaginary parts: chunk + 4,
      // i.e. ^ 64); boff[o] = the real-part K word of output o (0: real, 1: imaginary) in the
      // hi tile (the imaginary-part K word: the next chunk, i.e. ^ 16)
      uint32_t aoff[2], boff[2][2], msk[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int v = warp + j * kHProducerWarps;
        int eA = 0, rA = 0;
        bool cj = false;
        if (v < nv) {
          const int b1 = v % nb;
          if (v < nb) {
            eA = g.sa0 + hblk_index(g.ba0, kr.A[0], g.s, b1, nb);
            rA = g.ba0.row0 + (eA - g.sa0);
            cj = kr.A[0].conj != 0;
          } else {
            eA = g.sa1 + hblk_index(g.ba1, kr.A[1], g.s, b1, nb);
            rA = g.ba1.row0 + (eA - g.sa1);
            cj = kr.A[1].conj != 0;
          }
        }
        aoff[j] = (uint32_t)eA * 512u + (uint32_t)(lane >> 3) * 128u + (lane & 1) * 8 +
                  ((uint32_t)(((lane & 7) >> 1) ^ (rA & 7)) << 4);
        // real output: K_re <- A_r, K_im <- -A_i (conj A: +A_i); imaginary output: K_re <- A_i
        // (conj: -A_i), K_im <- A_r
        msk[j] = cj ? 0u : 0x80008000u;
        const int q = lane >> 2;                       // MMA group of the lane's centres
        const uint32_t atom = (uint32_t)(q >> 2) * atom_bytes, within = (lane & 3) * 4;
        const int ch = 2 * (q & 3);
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          const int n = 2 * v + o;
          boff[j][o] = atom + (uint32_t)(n >> 3) * 1024u + (uint32_t)(n & 7) * 128u + within +
                       ((uint32_t)(ch ^ (n & 7)) << 4);
        }
      }
      float accD[16];  // FP32 sums of the promoted partials: this row, 16 columns
      const bool has_cols = qq * 16 < npad;
      // Software pipeline over the stages (k = this stage):
      //  * the partial sum of stage k - 2 is read out of TMEM at the end of this stage
      //    (tcgen05.ld issued there, waited for after the first half of the next stage's rows),
      //    then its D buffer is released, before the MMAs of stage k are signalled;
      //  * the rows of stage k - 1 were stored into TMEM at the end of the previous iteration;
      //    their completion is awaited (and the MMA warp signalled) only after the first half
      //    of this stage's rows is formed, so the store latency is hidden behind that work.
      // The MMAs of stage k - 1 thus start one iteration late, which the three A/B slots absorb.
      auto promote_issue = [&](long long gg, uint32_t* v) {
        const int buf = (int)(gg & 1);
        wait(&dfull[buf], (uint32_t)((gg >> 1) & 1));
        tc_fence_after();
        if (has_cols) tmem_ld16(tmem + ((uint32_t)(grp * 32) << 16) + buf * 64 + qq * 16, v);
      };
      auto promote_finish = [&](long long gg, const uint32_t* v) {
        if (has_cols) {
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) accD[j] += __uint_as_float(v[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dempty[(int)(gg & 1)]);
      };
      auto publish = [&](int slot) {  // the rows (TMEM) and columns (shared) of a slot are complete
        tmem_wait_st();
        fence_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ab_full[slot]);
      };
      // the wave's segments in order, runs of consecutive segments with the same output slot
      // accumulated together (the patches of one survey form one run): one pipeline drain and
      // one epilogue per run
      for (int si = 0; si < args.plan.nseg;) {
      const int slot = args.plan.seg[si].slot;
      int nstage = 0;
      for (; si < args.plan.nseg && args.plan.seg[si].slot == slot; ++si)
        nstage += (seg_live(args.plan.seg[si]) + kHCentres - 1) / kHCentres;
#pragma unroll
      for (int j = 0; j < 16; ++j) accD[j] = 0.f;
      int prev_slot = 0;
      uint32_t pv[16];  // a partial sum on its way out of TMEM: read at the end of one stage,
                        // added in the middle of the next
      for (int k = 0; k < nstage; ++k) {
        wait(&in_full[islot], iph);
        wait(&ab_empty[aslot], aph ^ 1u);
        tc_fence_after();
        const uint32_t st = in_addr + (uint32_t)islot * in_bytes;
        const uint32_t bt = b_addr + (uint32_t)aslot * bslot_bytes;
        // B operand: the real embedding of A(Th1), fp16 hi and lo tiles
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (warp + j * kHProducerWarps >= nv) break;
          uint32_t arh, arl, aih, ail;
          split_h2(lds_64(st + aoff[j]), arh, arl);
          split_h2(lds_64(st + (aoff[j] ^ 64u)), aih, ail);
          const uint32_t m1 = msk[j], m2 = msk[j] ^ 0x80008000u;
          const uint32_t r0 = bt + boff[j][0], r1 = bt + boff[j][1], lt = 2 * atom_bytes;
          sts_32(r0, arh);
          sts_32(r0 ^ 16u, aih ^ m1);
          sts_32(r1, aih ^ m2);
          sts_32(r1 ^ 16u, arh);
          sts_32(r0 + lt, arl);
          sts_32((r0 ^ 16u) + lt, ail ^ m1);
          sts_32(r1 + lt, ail ^ m2);
          sts_32((r1 ^ 16u) + lt, arl);
        }
        // A operand (TMEM): this row's Khatri-Rao values for the warp's 16 centres, in two
        // groups of 8; the previous stage is published between them
        const uint32_t PB = st + xB0, PC = st + xC0;
        const uint32_t acol = tmem + ((uint32_t)(grp * 32) << 16) + kHDCols + aslot * kHACols + qq * 16;
        {
          uint32_t hi[8], lo[8];
          if (cjC) kr_group<true>(PB, PC, 0, hi, lo);
          else kr_group<false>(PB, PC, 0, hi, lo);
          if (k >= 3) promote_finish(gs + k - 3, pv);
          if (k >= 1) publish(prev_slot);
          tmem_st8(acol, hi);
          tmem_st8(acol + 64, lo);
        }
        {
          uint32_t hi[8], lo[8];
          if (cjC) kr_group<true>(PB, PC, 1, hi, lo);
          else kr_group<false>(PB, PC, 1, hi, lo);
          // every value this warp loaded from the staged stage has been used: it can be refilled
          __syncwarp();
          if (lane == 0) mbar_arrive(&in_empty[islot]);
          tmem_st8(acol + 8, hi);
          tmem_st8(acol + 64 + 8, lo);
        }
        if (k >= 2) promote_issue(gs + k - 2, pv);
        prev_slot = aslot;
        if (++islot == S_in) { islot = 0; iph ^= 1u; }
        if (++aslot == kHSlots) { aslot = 0; aph ^= 1u; }
      }
      // drain the pipeline: the partial sum read at the end of the last stage, the last
      // stage's rows, then the last two partial sums
      if (nstage >= 3) promote_finish(gs + nstage - 3, pv);
      if (nstage >= 1) publish(prev_slot);
      for (long long gg = gs + (nstage >= 2 ? nstage - 2 : 0); gg < gs + nstage; ++gg) {
        promote_issue(gg, pv);
        promote_finish(gg, pv);
      }
      gs += nstage;
      // ---------------------------------------------------------------- epilogue
      if (row_ok && has_cols && nstage > 0) {  // (an empty run adds nothing)
        const int pr = rr % npairs, nx = 2 * N + 3;
        const int kx = h_scale_exp(args.rowmax[g.bx.row0 + (eB - g.sx)]);
        const int kc = h_scale_exp(args.rowmax[g.bc.row0 + (eC - g.sc)]);
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int n = qq * 16 + j;
          if (n < ncols) {
            const int ga = n / (2 * nb), b1 = (n >> 1) % nb;
            const int mu = ga ? kr.mu[1] : kr.mu[0];
            const int arow = ga ? g.ba1.row0 + hblk_index(g.ba1, kr.A[1], g.s, b1, nb)
                                : g.ba0.row0 + hblk_index(g.ba0, kr.A[0], g.s, b1, nb);
            const double unscale = h_pow2d(-(kx + kc + h_scale_exp(args.rowmax[arow])));
            const size_t o = ((((size_t)mu * nx + (n2 + N + 1)) * nx + (n3 + N + 1)) * nb + b1) * npairs + pr;
            double* p = args.red + (size_t)slot * args.red_stride + 2 * o;
            p[0] += (double)accD[j] * unscale;
            p[1] += (double)accD[j + 1] * unscale;
          }
        }
      }
      }  // runs of segments
    }
  } else if (warp == kHWarpMma) {
    // ---------------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint64_t dbase = desc_sw128(saddr(sm));
      int aslot = 0;
      uint32_t aph = 0;
      long long gs = 0;
      for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
        const KRType kr = kKR[args.items[it].x];
        const int npad = (2 * kr.nmu * nb + 15) / 16 * 16;
        const uint32_t id = idesc(0u, npad);  // fp16 A and B, FP32 D
        for (int si = 0; si < args.plan.nseg; ++si) {
        const int nstage = (seg_live(args.plan.seg[si]) + kHCentres - 1) / kHCentres;
        for (int k = 0; k < nstage; ++k, ++gs) {
          const int buf = (int)(gs & 1);
          if (gs >= 2) wait(&dempty[buf], (uint32_t)(((gs >> 1) - 1) & 1));
          wait(&ab_full[aslot], aph);
          tc_fence_after();
          const uint32_t d = tmem + buf * 64;
          const uint32_t ah = tmem + kHDCols + aslot * kHACols, al = ah + 64;
          // descriptor of the slot's hi tile: start-address field (address / 16) plus the
          // offset / 16 (no carry: shared addresses stay below 2^18)
          const uint64_t db = dbase + (uint64_t)((aslot * bslot_bytes) >> 4);
          const uint64_t dl = (uint64_t)((2 * atom_bytes) >> 4);
#pragma unroll
          for (int q = 0; q < 8; ++q) {  // K = 16 halves = 8 centres per MMA
            const uint64_t bh = db + (uint64_t)((((q >> 2) * atom_bytes) + (q & 3) * 32) >> 4);
            mma_f16(d, ah + q * 8, bh, id, q > 0 ? 1u : 0u);
            mma_f16(d, ah + q * 8, bh + dl, id, 1u);
            mma_f16(d, al + q * 8, bh, id, 1u);
          }
          mma_commit(&ab_empty[aslot]);
          mma_commit(&dfull[buf]);
          if (++aslot == kHSlots) { aslot = 0; aph ^= 1u; }
        }
        }  // segments
      }
      // every MMA of this CTA has completed before the TMEM is released (also when a wait
      // above gave up); an MMA always finishes, so this bound is generous
      mma_commit(drain);
      if (!mbar_wait(drain, 0u, 4000000000LL)) err = 1;
    }
    __syncwarp();
  } else if (warp == kHWarpLoad) {
    // ---------------------------------------------------------------------- bulk-copy loader
    // One thread: per stage the four blocks of the item, each a contiguous range of the
    // stage-major wave array, copied with one cp.async.bulk each.
    if (lane == 0) {
      int islot = 0;
      uint32_t iph = 0;
      int last[kHMaxIn];  // parity of the last phase issued per slot (-1: none)
      for (int k = 0; k < kHMaxIn; ++k) last[k] = -1;
      for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
        const KRType kr = kKR[args.items[it].x];
        const HGeo g = hgeo(args, args.items[it], kr);
        const HBlk blk[4] = {g.bx, g.bc, g.ba0, g.ba1};
        const int srow[4] = {g.sx, g.sc, g.sa0, g.sa1};
        bool ok = g.sa1 + g.ba1.len <= args.stage_rows;
        for (int b = 0; b < 4; ++b)
          ok = ok && (blk[b].len == 0 || (blk[b].row0 >= 0 && blk[b].row0 + blk[b].len <= args.rows));
        if (!ok) {  // never for the supported shapes
          *abort_flag = 1;
          err = 1;
        }
        const uint32_t bytes = (uint32_t)(g.sa1 + g.ba1.len) * 512u;
        for (int si = 0; si < args.plan.nseg; ++si) {
        const WaveSeg& sgm = args.plan.seg[si];
        const int nstage = (seg_live(sgm) + kHCentres - 1) / kHCentres, kst0 = sgm.off / kHCentres;
        for (int k = 0; k < nstage; ++k) {
          wait(&in_empty[islot], iph ^ 1u);
          if (!*abort_flag) {  // nothing more is copied once the CTA gives up
            last[islot] = (int)iph;
            mbar_expect_tx(&in_full[islot], bytes);
            unsigned char* st = in_base + (size_t)islot * in_bytes;
            const float* src = args.wave + (size_t)(kst0 + k) * args.rows * 128;
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (blk[b].len > 0)
                bulk_load(st + srow[b] * 512, src + (size_t)blk[b].row0 * 128, (uint32_t)blk[b].len * 512u,
                          &in_full[islot]);
          }
          if (++islot == S_in) { islot = 0; iph ^= 1u; }
        }
        }  // segments
      }
      // every copy has landed before the shared memory is given up: the phases of a slot
      // complete in order, so its last issued phase covers the earlier ones
      for (int k = 0; k < S_in; ++k)
        if (last[k] >= 0 && !mbar_wait(&in_full[k], (uint32_t)last[k], 4000000000LL)) err = 1;
    }
    __syncwarp();
  }
  if (err) atomicExch(args.status, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kHTmemCols) : "memory");
}

// rows per staged stage: the x~B and C blocks of at most the tile's n2 values (128 rows =
// 128 / pairs values of n2, +2 for misalignment, at most 2N + 3) and two A blocks
int h_stage_rows(int nb, int N) {
  int rows = 128 / (nb * (nb + 1) / 2) + 2;
  if (rows > 2 * N + 3) rows = 2 * N + 3;
  return 2 * rows * nb + 2 * nb;
}
int h_npad_max(int nb) { return (4 * nb + 15) / 16 * 16; }
size_t h_fixed_smem(int nb) { return (size_t)kHSlots * 4 * h_npad_max(nb) * 128 + 1024 + 512; }
int h_in_stages(int nb, int N) {
  const size_t per = (size_t)h_stage_rows(nb, N) * 512;
  const size_t room = 227 * 1024 - h_fixed_smem(nb);
  int k = (int)(room / per);
  if (k > kHMaxIn) k = kHMaxIn;
  return k >= 2 ? k : 0;
}
size_t h_smem_bytes(int nb, int N) {
  return h_fixed_smem(nb) + (size_t)h_in_stages(nb, N) * h_stage_rows(nb, N) * 512;
}

}  // namespace

int h16_wave_rows(const Layout& L) { return (kXBTypes * (2 * L.N + 3) + L.nG + 4 * L.N + 1) * L.nb; }
static int h16_wave_pitch(int T) { return (T + kHCentres - 1) / kHCentres * kHCentres; }

bool h16_supported(const Layout& L) {
  return L.nb >= 1 && 4 * L.nb <= 64 && h_in_stages(L.nb, L.N) >= 2;
}
size_t contract_h16_wave_bytes(const Layout& L, int T) {
  return (size_t)h16_wave_rows(L) * h16_wave_pitch(T) * sizeof(float2);
}
size_t contract_h16_rowmax_bytes(const Layout& L) { return (size_t)h16_wave_rows(L) * sizeof(unsigned); }

cudaError_t contract_wave_h16(const Layout& L, const float2* rec, const float2* xw, const WavePlan& plan,
                              double* red, const int4* items, int n_items, float2* wave, unsigned* rowmax,
                              int* status, long long timeout, cudaStream_t s) {
  if (plan.total <= 0 || plan.nseg <= 0) return cudaSuccess;
  for (int i = 0; i < plan.nseg; ++i)  // segments start at stage boundaries
    if (plan.seg[i].off % kHCentres != 0) return cudaErrorInvalidValue;
  const int rows = h16_wave_rows(L), pitch = h16_wave_pitch(plan.total);
  const int row_g = kXBTypes * (2 * L.N + 3) * L.nb, row_w = row_g + L.nG * L.nb;
  cudaError_t e = cudaMemsetAsync(rowmax, 0, (size_t)rows * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  hwave_rowmax_kernel<<<dim3((rows + 31) / 32, (plan.total + 127) / 128), 256, 0, s>>>(L, rec, xw, plan, row_g,
                                                                                     row_w, rows, rowmax);
  hwave_transpose_kernel<<<dim3((rows + 31) / 32, pitch / 32), 256, 0, s>>>(
      L, rec, xw, plan, row_g, row_w, rows, rowmax, reinterpret_cast<float*>(wave));
  g_launches += 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  HArgs a;
  a.L = L; a.plan = plan; a.red = red; a.red_stride = tc_reduced_doubles(L);
  a.npairs = L.nb * (L.nb + 1) / 2;
  a.items = items; a.n_items = n_items;
  a.row_g = row_g; a.row_w = row_w;
  a.rowmax = rowmax;
  a.wave = reinterpret_cast<const float*>(wave);
  a.rows = rows;
  a.in_stages = h_in_stages(L.nb, L.N);
  a.stage_rows = h_stage_rows(L.nb, L.N);
  a.npad_max = h_npad_max(L.nb);
  a.timeout = timeout; a.status = status;
  if (a.in_stages < 2) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = h_smem_bytes(L.nb, L.N);
  e = cudaFuncSetAttribute(contract_h16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contract_h16_kernel<<<sms, kHThreads, smem, s>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ext4pcf
