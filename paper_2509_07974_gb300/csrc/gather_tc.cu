// Tensor-core neighbour gather (tcgen05, sm_103a) for the mixed-precision forms.
//
// Per centre and radial bin the record holds sums over the bin's pairs of a weight times a
// power of u = e^{i phi}: G (x u^n), XX (x^2 u^n), W (w u^m), XA (|x|^2 u^m), WW (w^2 u^m)
// and five triple terms (paper Eq. 4PCFUpsilon0 ff., Table tab:4PCFMCCorr).  Writing
// n = r + 3a or n = r - 3a with r in {-1, 0, 1} and 0 <= a < A splits every such sum into
// an outer product over the pairs:
//   sum_j (omega_j u_j^r) (u_j^{3a})   and   sum_j (omega_j u_j^r) conj(u_j^{3a}),
// and both follow from the four real sums Re/Im(omega u^r) x Re/Im(u^{3a}).  So per bin
//   D[row][col] = sum_j F_j[row] P_j[col]
// is a GEMM with K along the pairs, where the 39 feature rows F are Re/Im of omega u^r for
// omega in {x, x^2, w, |x|^2, w^2} (r = -1, 0, 1), x^3 (r = -1, 1), |x|^2 x (r = -1, 0) and
// w^3 (r = 0), and the columns P are Re/Im u^{3a}.
//
// Mapping onto tcgen05.mma (kind::tf32, M = 128, N = 2A rounded up to 16, K = 8 pairs):
//   * A operand (TMEM): feature row = TMEM lane (lanes 0..38 used), one column per pair.
//     Per K-block of 32 pairs the features are formed pair-per-lane, transposed through
//     shared memory and written row-per-lane with tcgen05.st.
//   * B operand (shared memory, K-major, 128-byte swizzle): u^{3a} per pair.
//   * 3xTF32: hi*hi + hi*lo + lo*hi, hi the top 10 mantissa bits, lo = x - hi.
//   * D (TMEM, FP32): two buffers of 128 / N independent sub-accumulators that the MMAs
//     rotate over (so that consecutive MMAs do not wait on each other's accumulation);
//     every 64 pairs of a bin the partial sum is read into
//     FP32 registers (long FP32 accumulation inside the tensor core loses bits), and at the
//     end of the bin's pairs in a chunk the registers are combined into the record.
// Warp roles during the accumulation: three generator groups of four warps (each group
// owns one pipeline stage: two feature warps and two power warps), two epilogue warps
// (TMEM lanes 0..63), one MMA-issuing thread.  Classification and bucketing by bin (stable,
// deterministic) are shared with the CUDA-core gather and use all 16 warps.  Every
// mbarrier wait is bounded by a clock budget; on expiry the kernel records an error code
// and runs to its end.
#include <algorithm>

#include "common.cuh"
#include "gather_common.cuh"
#include "tc_ptx.cuh"

namespace ext4pcf {

namespace {

constexpr int kGThreads = 512;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGroups = 3;       // generator groups = pipeline stages
constexpr int kKB = 32;          // pairs per K-block
constexpr int kSegKB = 2;        // K-blocks per TMEM partial sum
constexpr int kXpRows = 40;      // feature rows staged per K-block (row 39 is zero)
constexpr int kXpStride = 36;    // words per staged feature row (32 pairs + 4)
constexpr int kEpiWarp = 12;     // epilogue warps 12 (lanes 0..31) and 13 (lanes 32..63)
constexpr int kMmaWarp = 14;
constexpr uint32_t kGTmemCols = 512;
constexpr int kDColsMax = 64;    // D columns (A <= 32 powers)
// Each D buffer holds 128 columns: 128 / NPC independent sub-accumulators that successive
// MMAs of a partial sum rotate over (MMAs into one accumulator serialise on the tensor
// core's latency; independent ones overlap).  The epilogue adds the sub-accumulators.
constexpr int kDBufCols = 128;
constexpr int kACol0 = 2 * kDBufCols;  // A stages: hi [0, 32) + lo [32, 64) each
constexpr unsigned kFullMask = 0xFFFFFFFFu;

// feature row pairs (2i: real part, 2i + 1: imaginary part): weight type and power r
//   types: 0 x, 1 x^2, 2 w, 3 |x|^2, 4 w^2, 5 x^3, 6 |x|^2 x, 7 w^3
__constant__ signed char kRowType[20] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 4, 4, 4, 5, 5, 6, 6, 7};
__constant__ signed char kRowR[20] = {-1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 1, -1, 0, 0};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// omega u^r for r in {-1, 0, 1}
__device__ __forceinline__ float2 times_ur(float2 w, float2 u, int r) {
  if (r == 0) return w;
  const float2 v = r > 0 ? u : make_float2(u.x, -u.y);
  return cmulf(w, v);
}

// record element of weight type t at power n in bin b, or -1 if the record does not hold it
__device__ __forceinline__ int record_index(const Layout& L, int t, int n, int b) {
  const int N = L.N;
  switch (t) {
    case 0: return (n >= -2 * N - 3 && n <= 2 * N - 1) ? L.G(n, b) : -1;
    case 1: return (n >= -2 * N - 6 && n <= 2 * N - 2) ? L.XX(n, b) : -1;
    case 2: return (n >= 0 && n <= 2 * N) ? L.W(n, b) : -1;
    case 3: return (n >= 0 && n <= 2 * N + 2) ? L.XA(n, b) : -1;
    case 4: return (n >= 0 && n <= 2 * N) ? L.WW(n, b) : -1;
    case 5: return n == -8 ? L.TR(0, b) : (n == -4 ? L.TR(1, b) : -1);
    case 6: return n == -4 ? L.TR(2, b) : (n == 0 ? L.TR(3, b) : -1);
    default: return n == 0 ? L.TR(4, b) : -1;
  }
}

// bounded wait that also gives up at once when another thread of the CTA has given up
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* b, uint32_t parity, long long budget,
                                             volatile int* abort_flag) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

struct GTcArgs {
  GatherArgs g;
  int npow;        // A: powers u^{3a}, a < A
  int cap;         // pairs per chunk
  int max_kb;      // K-block list capacity
  long long timeout;
  int* status;
};

template <int NPC>  // D columns: 2A rounded up to 16
__global__ void __launch_bounds__(kGThreads, 1)
gather_tc_kernel(const GTcArgs args, float2* __restrict__ rec, float2* __restrict__ xw) {
  constexpr int kThreads = kGThreads;
  constexpr int kWarps = kGWarps;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (saddr(smem_raw) & 1023)) & 1023);
  const GatherArgs& ga = args.g;
  const SortedCat& cat = ga.cat;
  const Layout L = ga.L;
  const int nb = ga.bins.nb, cap = args.cap, A = args.npow;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int btile = NPC * 128;  // bytes of one K-major tile (NPC rows of 32 tf32)

  unsigned char* btiles = sm;  // [kGroups][hi, lo][btile]
  float* xp = reinterpret_cast<float*>(btiles + kGroups * 2 * btile);  // [kGroups][kXpRows][kXpStride]
  float2* acc = reinterpret_cast<float2*>(xp + kGroups * kXpRows * kXpStride);
  int4* kbl = reinterpret_cast<int4*>(acc + L.rec);
  double* e2 = reinterpret_cast<double*>(kbl + args.max_kb);
  float* e2f = reinterpret_cast<float*>(e2 + 65);
  float* win = e2f + 65;
  int* off = reinterpret_cast<int*>(win + 65);  // [65] bin offsets of the chunk
  int* wcnt = off + 65;                          // [warps][64] per-warp bin counts / positions
  int* rstart = wcnt + kWarps * 64;
  int* rpre = rstart + kMaxRows;
  int* misc = rpre + kMaxRows + 1;
  uint64_t* bars = reinterpret_cast<uint64_t*>(misc + 8);  // 8-byte aligned: 202 + 64 kWarps ints above
  uint64_t* st_full = bars;
  uint64_t* st_empty = bars + kGroups;
  uint64_t* d_full = bars + 2 * kGroups;
  uint64_t* d_empty = d_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(d_empty + 2);
  float2* eu = reinterpret_cast<float2*>(tmem_slot + 2);
  float2* ex = eu + cap;
  float* ew = reinterpret_cast<float*>(ex + cap);
  signed char* cbin = reinterpret_cast<signed char*>(ew + cap);  // bin of each candidate of a chunk

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int k = 0; k < kGroups; ++k) {
      mbar_init(&st_full[k], 4 * 32);
      mbar_init(&st_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&d_full[k], 1);
      mbar_init(&d_empty[k], 64);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B tiles start at zero (columns 2A .. NPC are never written); bin edges and counters
  for (int k = tid; k < kGroups * 2 * btile / 4; k += kThreads) reinterpret_cast<uint32_t*>(btiles)[k] = 0u;
  for (int b = tid; b <= nb; b += kThreads) {
    e2[b] = ga.bins.e2[b]; e2f[b] = ga.bins.e2f[b]; win[b] = ga.win[b];
  }
  for (int k = tid; k < kWarps * 64; k += kThreads) wcnt[k] = 0;
  if (tid == 0) misc[4] = 0;  // abort flag
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM lanes 64..127 of the A stages are never written by the feature warps: zero them
  // once so that the unused rows of D stay finite
  if (warp == 2 || warp == 3) {
    uint32_t z[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) z[j] = 0u;
    const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + kACol0;
    for (int c = 0; c < kGroups * 64; c += 16) tmem_st16(base + c, z);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const long long budget = args.timeout;
  volatile int* abort_flag = misc + 4;
  int err = 0;
  long long gkb = 0;   // K-blocks issued by this CTA so far (stage phases)
  long long gseg = 0;  // TMEM partial sums so far (D buffer phases)
  const uint32_t idesc_g = idesc(2u, NPC);
  const double rmax = ga.bins.rmax * (1.0 + 1e-9) + 1e-12;
  const double cell = cat.cell;

  for (int c = blockIdx.x; c < ga.T; c += gridDim.x) {
    const int pi = ga.centres[c];
    const double pxi = cat.px[pi], pyi = cat.py[pi];
    const float4 Pi = cat.p4[pi];
    if (tid == 0) {
      const double xc = pxi - cat.x0, yc = pyi - cat.y0;
      int cy0 = (int)floor((yc - rmax) / cell), cy1 = (int)floor((yc + rmax) / cell);
      cy0 = max(cy0, 0); cy1 = min(cy1, cat.ncy - 1);
      int nr = 0, tot = 0;
      for (int cy = cy0; cy <= cy1 && nr < kMaxRows; ++cy) {
        const double lo = cy * cell, hi = lo + cell;
        const double gap = fmax(0.0, fmax(lo - yc, yc - hi));
        if (gap > rmax) continue;
        const double hw = sqrt(fmax(0.0, rmax * rmax - gap * gap));
        int cx0 = (int)floor((xc - hw) / cell), cx1 = (int)floor((xc + hw) / cell);
        cx0 = max(cx0, 0); cx1 = min(cx1, cat.ncx - 1);
        if (cx0 > cx1) continue;
        const int a = cat.cell_start[cy * cat.ncx + cx0];
        const int b = cat.cell_start[cy * cat.ncx + cx1 + 1];
        if (b <= a) continue;
        rstart[nr] = a; rpre[nr] = tot; tot += b - a; ++nr;
      }
      rpre[nr] = tot;
      misc[0] = nr; misc[1] = tot;
    }
    for (int k = tid; k < L.rec; k += kThreads) acc[k] = make_float2(0.f, 0.f);
    __syncthreads();
    const int nr = misc[0], total = misc[1];
    unsigned long long pairs_here = 0;

    for (int cpos = 0; cpos < total;) {
      // ---- classification and stable bucketing by bin of the next cap candidates
      const int cend = min(total, cpos + cap);
      bucket_chunk<float, kWarps>(cat, rstart, rpre, nr, cpos, cend, pxi, pyi, Pi, e2, e2f, win, nb, cbin, wcnt, off,
                                  [&](int dst, float ur, float ui, int q) {
                                    float xr, xi, ww;
                                    Pair<float>::load_x(cat, q, xr, xi, ww);
                                    eu[dst] = make_float2(ur, ui);
                                    ex[dst] = make_float2(xr, xi);
                                    ew[dst] = ww;
                                  });
      // ---- K-block list: per bin ceil(count / 32) blocks of consecutive pairs; partial sums
      // of kSegKB blocks.  Entry: (first pair, pairs, bin, flags | segment << 3) with flags
      // 1: first block of a partial sum, 2: last block of a partial sum, 4: last of the bin
      if (warp == 0) {
        const int b = lane;
        const int nk = b < nb ? (off[b + 1] - off[b] + kKB - 1) / kKB : 0;
        const int ns = (nk + kSegKB - 1) / kSegKB;
        int kpre = nk, spre = ns;  // inclusive warp scans
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int a1 = __shfl_up_sync(kFullMask, kpre, o), a2 = __shfl_up_sync(kFullMask, spre, o);
          if (lane >= o) { kpre += a1; spre += a2; }
        }
        const int k0 = kpre - nk, s0 = spre - ns;
        for (int i = 0; i < nk; ++i) {
          const int first = off[b] + i * kKB;
          const int len = min(kKB, off[b + 1] - first);
          const int fl = ((i % kSegKB) == 0 ? 1 : 0) | ((i % kSegKB) == kSegKB - 1 || i == nk - 1 ? 2 : 0) |
                         (i == nk - 1 ? 4 : 0);
          kbl[k0 + i] = make_int4(first, len, b, fl | ((s0 + i / kSegKB) << 3));
        }
        if (lane == 31) { misc[2] = kpre; misc[3] = spre; }
      }
      __syncthreads();
      const int nkb = misc[2], nseg = misc[3];
      // ---- pass 3: tensor-core accumulation
      if (warp < 4 * kGroups) {
        const int g = warp >> 2, role = warp & 3;
        const int j0 = (int)((g - (gkb % kGroups) + kGroups) % kGroups);
        float* xg = xp + g * kXpRows * kXpStride;
        unsigned char* bh = btiles + g * 2 * btile;
        const uint32_t acol = tmem + kACol0 + g * 64;
        for (int j = j0; j < nkb; j += kGroups) {
          const long long G = gkb + j;
          const uint32_t ph = (uint32_t)((G / kGroups) & 1);
          const int4 kb = kbl[j];
          if (!mbar_wait_ab(&st_empty[g], ph ^ 1u, budget, abort_flag)) err = 1;
          tc_fence_after();
          const bool valid = lane < kb.y;
          const int e = kb.x + (valid ? lane : 0);
          const float2 u = valid ? eu[e] : make_float2(1.f, 0.f);
          if (role < 2) {
            // features of this lane's pair, transposed through shared memory
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");  // the previous block was read
            const float2 x = valid ? ex[e] : make_float2(0.f, 0.f);
            const float w = valid ? ew[e] : 0.f;
            const float2 x2 = cmulf(x, x);
            const float a2 = x.x * x.x + x.y * x.y, w2 = w * w;
            if (role == 0) {
#pragma unroll
              for (int i = 0; i < 9; ++i) {
                const int t = i / 3, r = i % 3 - 1;
                const float2 om = t == 0 ? x : (t == 1 ? x2 : make_float2(w, 0.f));
                const float2 v = times_ur(om, u, r);
                xg[(2 * i) * kXpStride + lane] = v.x;
                xg[(2 * i + 1) * kXpStride + lane] = v.y;
              }
            } else {
              const float2 x3 = cmulf(x2, x), ax = make_float2(a2 * x.x, a2 * x.y);
#pragma unroll
              for (int i = 9; i < 20; ++i) {
                const int t = i < 15 ? 3 + (i - 9) / 3 : (i < 17 ? 5 : (i < 19 ? 6 : 7));
                const int r = i < 15 ? (i - 9) % 3 - 1 : (i == 15 ? -1 : (i == 16 ? 1 : (i == 17 ? -1 : 0)));
                const float2 om = t == 3 ? make_float2(a2, 0.f)
                                : t == 4 ? make_float2(w2, 0.f)
                                : t == 5 ? x3
                                : t == 6 ? ax
                                         : make_float2(w2 * w, 0.f);
                const float2 v = times_ur(om, u, r);
                xg[(2 * i) * kXpStride + lane] = v.x;
                xg[(2 * i + 1) * kXpStride + lane] = t == 7 ? 0.f : v.y;
              }
            }
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");  // all features staged
            // this lane's feature row for the 32 pairs, split into tf32 hi + lo
            const int row = 32 * role + lane;
            uint32_t vh[32], vl[32];
            if (row < kXpRows) {
              const float4* src = reinterpret_cast<const float4*>(xg + row * kXpStride);
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const float4 v = src[q];
                split_tf32(v.x, vh[4 * q], vl[4 * q]);
                split_tf32(v.y, vh[4 * q + 1], vl[4 * q + 1]);
                split_tf32(v.z, vh[4 * q + 2], vl[4 * q + 2]);
                split_tf32(v.w, vh[4 * q + 3], vl[4 * q + 3]);
              }
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) { vh[k] = 0u; vl[k] = 0u; }
            }
            const uint32_t ta = acol + ((uint32_t)(32 * role) << 16);
            tmem_st16(ta, vh);
            tmem_st16(ta + 16, vh + 16);
            tmem_st16(ta + 32, vl);
            tmem_st16(ta + 48, vl + 16);
            tmem_wait_st();
            tc_fence_before();
          } else {
            // powers u^{3a} of this lane's pair for a in [a0, a1), tf32 hi + lo, into the
            // K-major swizzled B tiles (row 2a: real part, 2a + 1: imaginary part)
            const int ah = (A + 1) >> 1;
            const int a0 = role == 2 ? 0 : ah, a1 = role == 2 ? ah : A;
            const float2 u3 = cmulf(cmulf(u, u), u);
            float2 p = make_float2(1.f, 0.f);
            {
              float2 bb = u3;
              for (int ee = a0; ee; ee >>= 1) {
                if (ee & 1) p = cmulf(p, bb);
                bb = cmulf(bb, bb);
              }
            }
            for (int a = a0; a < a1; ++a) {
              uint32_t h0, l0, h1, l1;
              split_tf32(p.x, h0, l0);
              split_tf32(p.y, h1, l1);
              const uint32_t o0 = sw128_word_off(2 * a, lane, NPC), o1 = sw128_word_off(2 * a + 1, lane, NPC);
              *reinterpret_cast<uint32_t*>(bh + o0) = h0;
              *reinterpret_cast<uint32_t*>(bh + o1) = h1;
              *reinterpret_cast<uint32_t*>(bh + btile + o0) = l0;
              *reinterpret_cast<uint32_t*>(bh + btile + o1) = l1;
              p = cmulf(p, u3);
            }
            fence_async_smem();
          }
          mbar_arrive(&st_full[g]);
        }
      } else if (warp == kEpiWarp || warp == kEpiWarp + 1) {
        // partial sums of this lane's feature row, read every kSegKB blocks; combined into
        // the record at the last block of each bin
        const int row = 32 * (warp - kEpiWarp) + lane;
        float racc[NPC];
#pragma unroll
        for (int k = 0; k < NPC; ++k) racc[k] = 0.f;
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp - kEpiWarp)) << 16);
        for (int j = 0; j < nkb; ++j) {
          const int4 kb = kbl[j];
          if (!(kb.w & 2)) continue;
          const long long S = gseg + (kb.w >> 3);
          const int d = (int)(S & 1);
          if (!mbar_wait_ab(&d_full[d], (uint32_t)((S >> 1) & 1), budget, abort_flag)) err = 1;
          tc_fence_after();
#pragma unroll
          for (int sub = 0; sub < kDBufCols / NPC; ++sub)
#pragma unroll
            for (int q = 0; q < NPC / 16; ++q) {
              uint32_t v[16];
              tmem_ld16(trow + d * kDBufCols + sub * NPC + 16 * q, v);
              tmem_wait_ld();
#pragma unroll
              for (int k = 0; k < 16; ++k) racc[16 * q + k] += __uint_as_float(v[k]);
            }
          tc_fence_before();
          mbar_arrive(&d_empty[d]);
          if (kb.w & 4) {
            // rows 2i (Re omega u^r) and 2i + 1 (Im) of one (type, r) sit in adjacent lanes:
            //   sum omega u^{r+3a}      = (D_rr - D_ii, D_ri + D_ir)   (real-part lane, a >= 0)
            //   sum omega u^r u^{-3a}   = (D_rr + D_ii, D_ir - D_ri)   (imaginary-part lane, a >= 1)
            const int b = kb.z, i = row >> 1;
            const bool re = (row & 1) == 0;
            const int t = i < 20 ? kRowType[i] : -1, r = i < 20 ? kRowR[i] : 0;
#pragma unroll
            for (int a = 0; a < NPC / 2; ++a) {
              const float o0 = racc[2 * a], o1 = racc[2 * a + 1];
              const float p0 = __shfl_xor_sync(kFullMask, o0, 1), p1 = __shfl_xor_sync(kFullMask, o1, 1);
              if (t < 0 || a >= A) continue;
              float vr, vi;
              int n;
              if (re) {  // own = (D_rr, D_ri), partner = (D_ir, D_ii)
                vr = o0 - p1; vi = o1 + p0; n = r + 3 * a;
              } else {   // own = (D_ir, D_ii), partner = (D_rr, D_ri)
                if (a == 0) continue;
                vr = p0 + o1; vi = o0 - p1; n = r - 3 * a;
              }
              const int idx = record_index(L, t, n, b);
              if (idx >= 0) {
                float2 cur = acc[idx];
                cur.x += vr;
                cur.y += vi;
                acc[idx] = cur;
              }
            }
#pragma unroll
            for (int k = 0; k < NPC; ++k) racc[k] = 0.f;
          }
        }
      } else if (warp == kMmaWarp) {
        if (lane == 0) {
          for (int j = 0; j < nkb; ++j) {
            const int4 kb = kbl[j];
            const long long G = gkb + j;
            const int s = (int)(G % kGroups);
            const long long S = gseg + (kb.w >> 3);
            const int d = (int)(S & 1);
            if (kb.w & 1) {
              if (!mbar_wait_ab(&d_empty[d], (uint32_t)(((S >> 1) & 1) ^ 1), budget, abort_flag)) err = 1;
            }
            if (!mbar_wait_ab(&st_full[s], (uint32_t)((G / kGroups) & 1), budget, abort_flag)) err = 1;
            tc_fence_after();
            constexpr int nacc = kDBufCols / NPC;
            const uint32_t dcol = tmem + d * kDBufCols;
            const uint32_t a0 = tmem + kACol0 + s * 64;
            const uint32_t b0 = saddr(btiles + s * 2 * btile);
            const bool fresh = (kb.w & 1) != 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // K = 8 pairs per MMA: hi*hi + hi*lo + lo*hi
              const uint64_t dh = desc_sw128(b0 + q * 32), dl = desc_sw128(b0 + btile + q * 32);
              const int i0 = 3 * q;  // MMA i accumulates into sub-accumulator i % nacc
              mma_tf32(dcol + ((i0) % nacc) * NPC, a0 + q * 8, dh, idesc_g, (fresh && i0 < nacc) ? 0u : 1u);
              mma_tf32(dcol + ((i0 + 1) % nacc) * NPC, a0 + q * 8, dl, idesc_g, (fresh && i0 + 1 < nacc) ? 0u : 1u);
              mma_tf32(dcol + ((i0 + 2) % nacc) * NPC, a0 + 32 + q * 8, dh, idesc_g,
                       (fresh && i0 + 2 < nacc) ? 0u : 1u);
            }
            mma_commit(&st_empty[s]);
            if (kb.w & 2) mma_commit(&d_full[d]);
          }
        }
        __syncwarp();
      }
      gkb += nkb;
      gseg += nseg;
      __syncthreads();
      pairs_here += (unsigned long long)off[nb];
      cpos = cend;
      __syncthreads();
    }
    // ---- the record
    float2* dst = rec + (size_t)c * L.rec;
    for (int k = tid; k < L.rec; k += kThreads) dst[k] = acc[k];
    if (tid == 0) {
      float xr, xi, ww;
      Pair<float>::load_x(cat, pi, xr, xi, ww);
      xw[2 * (size_t)c] = make_float2(xr, xi);
      xw[2 * (size_t)c + 1] = make_float2(ww, 0.f);
      atomicAdd(ga.pair_count, pairs_here);
    }
    __syncthreads();
  }
  if (err) atomicExch(args.status, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols) : "memory");
}

int gtc_npow(int N) {
  // powers u^{3a}, a < A: r + 3a and r - 3a (r in {-1, 0, 1}) must reach 2N + 6, and the
  // triple terms need u^-8 (a = 3)
  const int A = (2 * N + 5 + 2) / 3 + 1;
  return A < 4 ? 4 : A;
}

size_t gtc_fixed_bytes(const Layout& L, int npc, int max_kb) {
  return (size_t)kGroups * 2 * npc * 128 + (size_t)kGroups * kXpRows * kXpStride * 4 + (size_t)L.rec * 8 +
         (size_t)max_kb * 16 + 65 * 8 + 2 * 65 * 4 + (65 + kGWarps * 64 + 2 * kMaxRows + 1 + 8) * 4 +
         10 * 8 + 8 + 1024;
}

}  // namespace

bool gather_tc_supported(const Layout& L) {
  return L.nb >= 1 && L.nb <= 32 && 2 * gtc_npow(L.N) <= kDColsMax &&
         gtc_fixed_bytes(L, kDColsMax, 8192 / kKB + 33) + 21 * kGThreads <= 227 * 1024;
}

cudaError_t gather_wave_tc(const SortedCat& cat, const Bins& bins, const Layout& L, const int* centres, int T,
                           float2* rec, float2* xw, unsigned long long* pair_count, int sm_count, int* status,
                           long long timeout, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  GTcArgs a;
  a.g.cat = cat; a.g.bins = bins; a.g.L = L; a.g.centres = centres; a.g.T = T; a.g.pair_count = pair_count;
  for (int b = 0; b <= bins.nb; ++b) {
    const double e = sqrt(bins.e2[b]);
    const double err = 4.0 * 1.2e-7 * (cat.cell + e);
    a.g.win[b] = (float)(2.0 * e * err + err * err);
  }
  a.g.mb = 0; a.g.nblk = 0; a.g.cap = 0;
  a.npow = gtc_npow(L.N);
  const int npc = 2 * a.npow <= 32 ? 32 : 64;  // the kernel's D width (template argument)
  // every wait inside the kernel is short (microseconds); 2e8 cycles (~0.1 s) bounds one
  a.timeout = std::min<long long>(timeout, 200000000LL);
  a.status = status;
  // chunk capacity: what the shared memory leaves, in multiples of the CTA size
  const size_t budget = 227 * 1024;
  int cap = 8192;
  for (;;) {
    const int max_kb = cap / kKB + L.nb + 1;
    const size_t need = gtc_fixed_bytes(L, npc, max_kb) + (size_t)cap * 21;
    if (need <= budget || cap <= kGThreads) break;
    cap -= kGThreads;
  }
  a.cap = cap;
  a.max_kb = cap / kKB + L.nb + 1;
  const size_t smem = gtc_fixed_bytes(L, npc, a.max_kb) + (size_t)cap * 21;
  if (smem > budget) return cudaErrorInvalidConfiguration;
  const int grid = std::min(T, sm_count > 0 ? sm_count : 148);
  cudaError_t e;
  if (npc <= 32) {
    e = cudaFuncSetAttribute(gather_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gather_tc_kernel<32><<<grid, kGThreads, smem, s>>>(a, rec, xw);
  } else {
    e = cudaFuncSetAttribute(gather_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gather_tc_kernel<64><<<grid, kGThreads, smem, s>>>(a, rec, xw);
  }
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ext4pcf
