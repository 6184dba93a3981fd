// Shared by the neighbour-gather kernels: the pair classification (bin decision and
// u = e^{i phi}) for FP64 and cell-anchored FP32 positions, and the launch arguments.
#pragma once
#include "common.cuh"

namespace ext4pcf {
namespace {

constexpr int kMaxRows = 64;  // rows of cells that can hold partners of one centre

__device__ __forceinline__ int bin_search(const double* e2, int nb, double r2) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (r2 >= e2[mid]) lo = mid; else hi = mid;
  }
  return lo;
}

// Exact FP64 decision, identical to the definition: two rounded products, one rounded sum.
__device__ __forceinline__ int classify_f64(double dx, double dy, const double* e2, int nb) {
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (!(r2 >= e2[0]) || !(r2 < e2[nb])) return -1;
  return bin_search(e2, nb, r2);
}

struct CentreF64 { double x, y; };

// Bin lookup of the FP32 decision.  The squared edges e2f[0..nb] are floats >= 0, whose bit
// patterns increase with their values; tab[i] is the bin of the float with bits
// base + (i << shift) (the largest b < nb with e2f[b] <= it), so for r2 in [e2f[0], e2f[nb])
// tab[(bits(r2) - base) >> shift] is at most the bin of r2, and a short forward walk over the
// edges ends at it.
struct BinLookup {
  const unsigned char* tab;  // [256], shared memory
  unsigned base;             // bits of e2f[0]
  int shift;                 // (bits(e2f[nb]) - base) >> shift < 256
  float out_lo, out_hi;      // r2 outside [out_lo, out_hi): no bin, whatever the rounding
};

// Returns the bin of candidate q (or -1) and u = e^{i phi}.
template <typename R> struct Pair;

template <> struct Pair<double> {
  __device__ static int classify(const SortedCat& cat, int q, double cx, double cy, const float4&,
                                 const double* e2, const float*, const float*, const BinLookup&, int nb,
                                 double& ur, double& ui) {
    double dx = cat.px[q] - cx, dy = cat.py[q] - cy;
    int b = classify_f64(dx, dy, e2, nb);
    if (b >= 0) {
      double rinv = 1.0 / sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
      ur = dx * rinv; ui = dy * rinv;
    }
    return b;
  }
  // u of a pair already classified into a bin (the same arithmetic as classify)
  __device__ static void direction(const SortedCat& cat, int q, double cx, double cy, const float4&, double& ur,
                                   double& ui) {
    double dx = cat.px[q] - cx, dy = cat.py[q] - cy;
    double rinv = 1.0 / sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    ur = dx * rinv; ui = dy * rinv;
  }
  __device__ static void load_x(const SortedCat& cat, int q, double& xr, double& xi, double& w) {
    xr = cat.xr[q]; xi = cat.xi[q]; w = cat.w[q];
  }
};

template <> struct Pair<float> {
  __device__ static int classify(const SortedCat& cat, int q, double cx, double cy, const float4& P,
                                 const double* e2, const float* e2f, const float* win, const BinLookup& lk,
                                 int nb, float& ur, float& ui) {
    float4 Q = cat.p4[q];
    float dx = (Q.x - P.x) + (Q.z - P.z);
    float dy = (Q.y - P.y) + (Q.w - P.w);
    float r2 = dx * dx + dy * dy;
    int b;
    // the float decision stands unless r2 is within the edge's rounding window
    if (r2 < lk.out_lo || r2 >= lk.out_hi) return -1;
    if (r2 < e2f[0]) {
      b = -1;
    } else if (r2 >= e2f[nb]) {
      b = nb;
    } else {
      b = lk.tab[min((__float_as_uint(r2) - lk.base) >> lk.shift, 255u)];
      while (b + 1 < nb && r2 >= e2f[b + 1]) ++b;
    }
    bool near = false;
    if (b < 0) near = true;  // within win[0] of the inner edge
    else if (b == nb) near = true;
    else near = (r2 - e2f[b] < win[b]) || (e2f[b + 1] - r2 <= win[b + 1]);
    if (near) b = classify_f64(cat.px[q] - cx, cat.py[q] - cy, e2, nb);
    if (b >= 0) {
      float rinv = rsqrtf(r2);
      ur = dx * rinv; ui = dy * rinv;
    }
    return b;
  }
  // u of a pair already classified into a bin (the same arithmetic as classify)
  __device__ static void direction(const SortedCat& cat, int q, double, double, const float4& P, float& ur,
                                   float& ui) {
    float4 Q = cat.p4[q];
    float dx = (Q.x - P.x) + (Q.z - P.z);
    float dy = (Q.y - P.y) + (Q.w - P.w);
    float rinv = rsqrtf(dx * dx + dy * dy);
    ur = dx * rinv; ui = dy * rinv;
  }
  __device__ static void load_x(const SortedCat& cat, int q, float& xr, float& xi, float& w) {
    float4 s = cat.s4[q];
    xr = s.x; xi = s.y; w = s.z;
  }
};

struct GatherArgs {
  SortedCat cat;
  Bins bins;
  Layout L;
  WavePlan plan;       // the wave's segments (centre lists, grids, record offsets)
  SortedCat cen;       // the galaxies' sorted arrays, where the centres are (cat: the neighbours,
                       // the galaxies or a reduced catalogue of the tree approximation)
  int accumulate;      // 0: write the records (and the centres' x, w); 1: add into them
  int cap;
  int mb;    // powers per warp block (<= MB)
  int nblk;  // power blocks
  unsigned long long* pair_count;
};

}  // namespace
}  // namespace ext4pcf

namespace ext4pcf {
namespace {

// Classifies the candidates [cpos, cend) of one centre (cend - cpos <= the capacity of
// cbin and of the pair arrays) and buckets its pairs by radial bin in a stable order (bin,
// then candidate index).  Warp w takes a contiguous slice of the candidates; pass 1 stores
// each candidate's bin (-1: outside every bin) and counts per (warp, bin); pass 2 recomputes
// u for the pairs and calls store(dst, ur, ui, q) with the pair's bucketed position dst and
// catalogue position q.  On return off[0..nb] holds the bin offsets (off[nb] = pairs).
// Candidate t maps to catalogue position rstart[r] + t - rpre[r] for the row r with
// rpre[r] <= t < rpre[r + 1].  Three block-wide barriers in all.
template <typename R, int NW, typename Store>
__device__ __forceinline__ void bucket_chunk(const SortedCat& cat, const int* rstart, const int* rpre, int nr,
                                             int cpos, int cend, double pxi, double pyi, const float4& Pi,
                                             const double* e2, const float* e2f, const float* win,
                                             BinLookup lk, int nb, signed char* cbin, int* wcnt, int* off,
                                             Store store) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xFFFFFFFFu, lt = (1u << lane) - 1u;
  const int ncand = cend - cpos;
  const int per = ((ncand + NW - 1) / NW + 31) & ~31;
  const int w0 = cpos + warp * per, w1 = min(cend, w0 + per);
  // row of this warp's first candidate (every lane starts there and walks forward)
  int r0 = 0;
  if (w0 < w1) {
    int lo = 0, hi = nr;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w0 >= rpre[mid]) lo = mid; else hi = mid;
    }
    r0 = lo;
  }
  if (lane < nb) wcnt[warp * 64 + lane] = 0;
  __syncwarp();
  lk.out_lo = e2f[0] - win[0];
  lk.out_hi = e2f[nb] + win[nb];
  // ---- pass 1: bin of every candidate, counts per (warp, bin)
  int r = r0;
  for (int t0 = w0; t0 < w1; t0 += 32) {
    const int t = t0 + lane;
    int b = -1;
    if (t < w1) {
      while (r + 1 < nr && t >= rpre[r + 1]) ++r;
      R ur, ui;
      b = Pair<R>::classify(cat, rstart[r] + (t - rpre[r]), pxi, pyi, Pi, e2, e2f, win, lk, nb, ur, ui);
      cbin[t - cpos] = (signed char)b;
    }
    const unsigned peers = __match_any_sync(full, b);
    if (b >= 0 && (peers & lt) == 0) wcnt[warp * 64 + b] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // ---- bin offsets and every warp's first position per bin
  if (warp == 0) {
    int tot = 0;
    if (lane < nb)
      for (int w = 0; w < NW; ++w) tot += wcnt[w * 64 + lane];
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane < nb) {
      int pos = inc - tot;
      off[lane] = pos;
      for (int w = 0; w < NW; ++w) {
        const int c = wcnt[w * 64 + lane];
        wcnt[w * 64 + lane] = pos;
        pos += c;
      }
    }
    if (lane == 31) off[nb] = inc;
  }
  __syncthreads();
  // ---- pass 2: u of every pair, written at its bucketed position
  r = r0;
  for (int t0 = w0; t0 < w1; t0 += 32) {
    const int t = t0 + lane;
    int b = -1, q = 0;
    if (t < w1) {
      while (r + 1 < nr && t >= rpre[r + 1]) ++r;
      b = cbin[t - cpos];
      q = rstart[r] + (t - rpre[r]);
    }
    const unsigned peers = __match_any_sync(full, b);
    if (b >= 0) {
      R ur, ui;
      Pair<R>::direction(cat, q, pxi, pyi, Pi, ur, ui);
      store(wcnt[warp * 64 + b] + __popc(peers & lt), ur, ui, q);
    }
    __syncwarp();
    if (b >= 0 && (peers & lt) == 0) wcnt[warp * 64 + b] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
}

}  // namespace
}  // namespace ext4pcf
