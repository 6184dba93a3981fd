// Neighbour gather: for each centre galaxy i of a wave, the spin-weighted multipoles
//   G_n(theta_i, Theta) = sum_j x_j e^{i n phi_ij},   x_j = w_j gamma_c,j
// of its neighbours in every radial bin, plus W_n and the quantities that the
// multiple-counting corrections need (paper Eq. 4PCFUpsilon0 ff., Table tab:4PCFMCCorr).
//
// One CTA (8 warps) per centre:
//   (a) the rows of cells that can hold partners are contiguous ranges of the cell-sorted
//       catalogue (found by one warp, a row per lane); the CTA streams them, keeps pairs
//       with Theta_lo^2 <= r^2 < Theta_hi^2, and buckets them by radial bin into a
//       shared-memory chunk (stable order, so the summation order is deterministic).  Chunks
//       hold up to `cap` candidates; long neighbour lists take several chunks.
//   (b) the work of a chunk is split into items (bin, power block): block k holds the powers
//       m in [k*mb, k*mb+mb) of u = e^{i phi_ij}.  The warps take the items in turn, outer
//       bins first.  For an item each lane walks pairs of the bin, raises u to the block's
//       first power (u^mb is stored per pair) and steps through the block by recurrence in
//       registers, accumulating seven real weights times u^m: Re x, Im x, Re x^2, Im x^2, w,
//       |x|^2, w^2.  The complex sums x u^{+-m} and x^2 u^{+-m} follow from the first four.
//       The 32 lanes' partial sums are combined by a transposed butterfly (each lane ends
//       with V/32 totals) and added to the centre's record in shared memory; no two items
//       of a chunk share a record entry.
//   (c) the triple terms, split over the power blocks in FP32, are summed in block order,
//       and the record is written to the wave buffer (or added to it, for the later passes
//       of the tree approximation).
// FP64 variant: positions and arithmetic in double; the bin decision r^2 = dx*dx + dy*dy is
// evaluated with two rounded products and one rounded sum, as the FP64 definition reads.
// FP32 variant: positions are cell-anchored floats (cell offset exact, in-cell offset
// rounded), so dx is accurate to ~1e-7 of the cell size; pairs whose r^2 lies within a few
// rounding errors of a bin edge are re-decided from the double positions.
#include "common.cuh"
#include "gather_common.cuh"

namespace ext4pcf {

namespace {

constexpr int kThreads = 256;
// FP32 (6-power blocks) splits the triple terms over the power blocks: partial sums per
// (bin, block) in shared memory, added in block order at the end of the centre
template <typename R, int MB> constexpr bool kTrSplitOf = sizeof(R) == 4 && MB >= 6;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Bucketed pairs in shared memory, structure of arrays: uv = (u_re, u_im, v_re, v_im) with
// u = e^{i phi}, v = u^mb; x = w gamma_c; w.  28 bytes per pair in FP32.
template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
struct __align__(16) Dbl4 { double x, y, z, w; };
template <> struct Vec4<double> { using T = Dbl4; };
template <typename R> struct EntArrays {
  typename Vec4<R>::T* uv;
  cplx_t<R>* x;
  R* w;
};

template <typename R, int MB> struct GCfg {
  static constexpr int kRaw = 14 * MB + 10;
  static constexpr int V = (kRaw + 31) / 32 * 32;
};

template <typename R>
__device__ __forceinline__ void cpow(R br, R bi, int e, R& pr, R& pi) {
  pr = R(1); pi = R(0);
  while (e) {
    if (e & 1) { R t = pr * br - pi * bi; pi = pr * bi + pi * br; pr = t; }
    R t = br * br - bi * bi; bi = R(2) * br * bi; br = t;
    e >>= 1;
  }
}

// u^e for 0 <= e < 32 by binary powering, unrolled (e is uniform across the warp)
template <typename R>
__device__ __forceinline__ void cpow5(R br, R bi, int e, R& pr, R& pi) {
  pr = R(1); pi = R(0);
#pragma unroll
  for (int bit = 0; bit < 5; ++bit) {
    if (e & (1 << bit)) { R t = pr * br - pi * bi; pi = pr * bi + pi * br; pr = t; }
    if (e >> (bit + 1)) { R t = br * br - bi * bi; bi = R(2) * br * bi; br = t; }
  }
}

// transposed butterfly: after the call lane l holds in a[0..V/32) the warp totals of the
// original slots j + base(l), base(l) = sum_k bit_k(l) * V / 2^(5-k)
template <typename R, int V, int OFF>
__device__ __forceinline__ void rt_step(R* a, int lane) {
  constexpr int H = V / 2;
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    R send = up ? a[j] : a[j + H];
    R keep = up ? a[j + H] : a[j];
    a[j] = keep + __shfl_xor_sync(kFull, send, OFF);
  }
}
template <typename R, int V>
__device__ __forceinline__ void reduce_transpose(R* a, int lane) {
  rt_step<R, V, 16>(a, lane);
  rt_step<R, V / 2, 8>(a, lane);
  rt_step<R, V / 4, 4>(a, lane);
  rt_step<R, V / 8, 2>(a, lane);
  rt_step<R, V / 16, 1>(a, lane);
}


// FP32 pass-3 inner loop with packed pairs: every (Re, Im) accumulator pair takes one
// two-lane fused multiply-add per pair of the bin (each lane rounds like a scalar FFMA), and
// the power recurrence u^{m+1} = u^m u runs on the pair (Re, Im) as one packed multiply and
// one packed multiply-add.  Fills a[0, 14 MB + 10) in the slot order of the scalar path.
template <int MB>
__device__ __forceinline__ void accumulate_f32x2(float* a, const float4* __restrict__ euv,
                                                 const float2* __restrict__ ex, const float* __restrict__ ew,
                                                 int s0, int s1, int lane, int k, int mb, bool first) {
  float2 acc[7 * MB];
#pragma unroll
  for (int j = 0; j < 7 * MB; ++j) acc[j] = make_float2(0.f, 0.f);
  float tr[10];
#pragma unroll
  for (int j = 0; j < 10; ++j) tr[j] = 0.f;
  for (int e0 = s0 + lane; e0 < s1; e0 += 64) {
    const int e1 = e0 + 32;
    const bool two = e1 < s1;
    const int e1c = two ? e1 : e0;
    const float4 q0 = euv[e0], q1 = euv[e1c];
    const float2 xx0 = ex[e0], xx1 = ex[e1c];
    const float w0 = ew[e0];
    // the second pair adds nothing when it is absent
    const float xr1 = two ? xx1.x : 0.f, xi1 = two ? xx1.y : 0.f, w1 = two ? ew[e1c] : 0.f;
    float2 P0, P1;
    cpow5<float>(q0.z, q0.w, k, P0.x, P0.y);
    cpow5<float>(q1.z, q1.w, k, P1.x, P1.y);
    const float2 U0 = make_float2(q0.x, q0.y), U0s = make_float2(-q0.y, q0.x);
    const float2 U1 = make_float2(q1.x, q1.y), U1s = make_float2(-q1.y, q1.x);
    const float wt0[7] = {xx0.x, xx0.y, xx0.x * xx0.x - xx0.y * xx0.y, 2.f * xx0.x * xx0.y, w0,
                          xx0.x * xx0.x + xx0.y * xx0.y, w0 * w0};
    const float wt1[7] = {xr1, xi1, xr1 * xr1 - xi1 * xi1, 2.f * xr1 * xi1, w1, xr1 * xr1 + xi1 * xi1, w1 * w1};
    auto step = [&](int t) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        acc[7 * t + q] = __ffma2_rn(make_float2(wt0[q], wt0[q]), P0, acc[7 * t + q]);
        acc[7 * t + q] = __ffma2_rn(make_float2(wt1[q], wt1[q]), P1, acc[7 * t + q]);
      }
      P0 = __ffma2_rn(make_float2(P0.x, P0.x), U0, __fmul2_rn(make_float2(P0.y, P0.y), U0s));
      P1 = __ffma2_rn(make_float2(P1.x, P1.x), U1, __fmul2_rn(make_float2(P1.y, P1.y), U1s));
    };
    if (mb == MB) {
#pragma unroll
      for (int t = 0; t < MB; ++t) step(t);
    } else {
#pragma unroll
      for (int t = 0; t < MB; ++t)
        if (t < mb) step(t);
    }
    if (first) {
      // x^3 u^-8, x^3 u^-4, x^2 x^* u^-4, x^2 x^*, w^3 (the second pair is zero if absent)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float ur = q ? q1.x : q0.x, ui = q ? q1.y : q0.y;
        const float* wt = q ? wt1 : wt0;
        const float xr = wt[0], xi = wt[1], x2r = wt[2], x2i = wt[3], ww = wt[4], xa = wt[5], w2 = wt[6];
        float u2r = ur * ur - ui * ui, u2i = 2.f * ur * ui;
        float u4r = u2r * u2r - u2i * u2i, u4i = 2.f * u2r * u2i;
        float u8r = u4r * u4r - u4i * u4i, u8i = 2.f * u4r * u4i;
        float x3r = x2r * xr - x2i * xi, x3i = x2r * xi + x2i * xr;
        float xcr = xa * xr, xci = xa * xi;  // x^2 x^* = |x|^2 x
        tr[0] += x3r * u8r + x3i * u8i;  // x3 * conj(u8)
        tr[1] += x3i * u8r - x3r * u8i;
        tr[2] += x3r * u4r + x3i * u4i;
        tr[3] += x3i * u4r - x3r * u4i;
        tr[4] += xcr * u4r + xci * u4i;
        tr[5] += xci * u4r - xcr * u4i;
        tr[6] += xcr;
        tr[7] += xci;
        tr[8] += w2 * ww;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 7 * MB; ++j) { a[2 * j] = acc[j].x; a[2 * j + 1] = acc[j].y; }
#pragma unroll
  for (int j = 0; j < 10; ++j) a[14 * MB + j] = tr[j];
}

// v^k for the block index k (uniform across the warp): the shortest product chain for
// k < 8 as straight-line code behind one uniform branch, binary powering beyond
__device__ __forceinline__ float2 cmul_f(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void vpow_block(float vr, float vi, int k, float2& P) {
  const float2 v = make_float2(vr, vi);
  switch (k) {
    case 0: P = make_float2(1.f, 0.f); return;
    case 1: P = v; return;
    case 2: P = cmul_f(v, v); return;
    case 3: P = cmul_f(cmul_f(v, v), v); return;
    case 4: { const float2 v2 = cmul_f(v, v); P = cmul_f(v2, v2); return; }
    case 5: { const float2 v2 = cmul_f(v, v); P = cmul_f(cmul_f(v2, v2), v); return; }
    case 6: { const float2 v2 = cmul_f(v, v); P = cmul_f(cmul_f(v2, v2), v2); return; }
    case 7: { const float2 v2 = cmul_f(v, v); P = cmul_f(cmul_f(cmul_f(v2, v2), v2), v); return; }
    default: cpow5<float>(vr, vi, k, P.x, P.y); return;
  }
}

// FP32 pass-3 inner loop, one pair per lane per iteration (for larger power blocks: the
// per-pair set-up -- loads, the block's first power, the weights -- is paid once per block
// of MB powers).  Fills a[0, 14 MB + 10) in the slot order of the scalar path.
template <int MB>
__device__ __forceinline__ void accumulate1_f32x2(float* a, const float4* __restrict__ euv,
                                                  const float2* __restrict__ ex, const float* __restrict__ ew,
                                                  int s0, int s1, int lane, int k, int mb, int tr_nsub) {
  float2 acc[7 * MB];
#pragma unroll
  for (int j = 0; j < 7 * MB; ++j) acc[j] = make_float2(0.f, 0.f);
  for (int e = s0 + lane; e < s1; e += 32) {
    const float4 q = euv[e];
    const float2 xx = ex[e];
    const float w = ew[e];
    float2 P;
    vpow_block(q.z, q.w, k, P);
    const float2 U = make_float2(q.x, q.y), Us = make_float2(-q.y, q.x);
    const float wt[7] = {xx.x, xx.y, xx.x * xx.x - xx.y * xx.y, 2.f * xx.x * xx.y, w,
                         xx.x * xx.x + xx.y * xx.y, w * w};
    auto step = [&](int t) {
#pragma unroll
      for (int qq = 0; qq < 7; ++qq) acc[7 * t + qq] = __ffma2_rn(make_float2(wt[qq], wt[qq]), P, acc[7 * t + qq]);
      P = __ffma2_rn(make_float2(P.x, P.x), U, __fmul2_rn(make_float2(P.y, P.y), Us));
    };
    if (mb == MB) {
#pragma unroll
      for (int t = 0; t < MB; ++t) step(t);
    } else {
#pragma unroll
      for (int t = 0; t < MB; ++t)
        if (t < mb) step(t);
    }
  }
#pragma unroll
  for (int j = 0; j < 7 * MB; ++j) { a[2 * j] = acc[j].x; a[2 * j + 1] = acc[j].y; }
  // x^3 u^-8, x^3 u^-4, x^2 x^* u^-4, x^2 x^*, w^3: a pass of its own (so that these sums
  // hold no registers in the power loop), shared by the tr_nsub power blocks of the bin:
  // block k takes the 32-pair groups k, k + tr_nsub, ...  The caller adds the blocks'
  // partial sums in a fixed order.
  float tr[10];
#pragma unroll
  for (int j = 0; j < 10; ++j) tr[j] = 0.f;
  {
    for (int e = s0 + lane + 32 * k; e < s1; e += 32 * tr_nsub) {
      const float4 q = euv[e];
      const float2 xx = ex[e];
      const float w = ew[e];
      const float ur = q.x, ui = q.y, xr = xx.x, xi = xx.y;
      const float x2r = xr * xr - xi * xi, x2i = 2.f * xr * xi, xa = xr * xr + xi * xi;
      float u2r = ur * ur - ui * ui, u2i = 2.f * ur * ui;
      float u4r = u2r * u2r - u2i * u2i, u4i = 2.f * u2r * u2i;
      float u8r = u4r * u4r - u4i * u4i, u8i = 2.f * u4r * u4i;
      float x3r = x2r * xr - x2i * xi, x3i = x2r * xi + x2i * xr;
      float xcr = xa * xr, xci = xa * xi;  // x^2 x^* = |x|^2 x
      tr[0] += x3r * u8r + x3i * u8i;  // x3 * conj(u8)
      tr[1] += x3i * u8r - x3r * u8i;
      tr[2] += x3r * u4r + x3i * u4i;
      tr[3] += x3i * u4r - x3r * u4i;
      tr[4] += xcr * u4r + xci * u4i;
      tr[5] += xci * u4r - xcr * u4i;
      tr[6] += xcr;
      tr[7] += xci;
      tr[8] += (w * w) * w;
    }
  }
#pragma unroll
  for (int j = 0; j < 10; ++j) a[14 * MB + j] = tr[j];
}

template <typename R, int MB, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
gather_kernel(const GatherArgs args, cplx_t<R>* __restrict__ rec, cplx_t<R>* __restrict__ xw) {
  using Cx = cplx_t<R>;
  constexpr int V = GCfg<R, MB>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  const SortedCat& cat = args.cat;
  const Layout L = args.L;
  const int nb = args.bins.nb, cap = args.cap, mb = args.mb, nblk = args.nblk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  using V4 = typename Vec4<R>::T;
  V4* euv = reinterpret_cast<V4*>(smem);
  Cx* ex = reinterpret_cast<Cx*>(euv + cap);
  R* ew = reinterpret_cast<R*>(ex + cap);
  double* e2 = reinterpret_cast<double*>(ew + cap);
  float* e2f = reinterpret_cast<float*>(e2 + 65);
  float* win = e2f + 65;
  int* off = reinterpret_cast<int*>(win + 65);  // [65] bin offsets of the chunk
  int* wcnt = off + 65;                          // [warps][64] per-warp bin counts / positions
  int* rstart = wcnt + kWarps * 64;
  int* rpre = rstart + kMaxRows;
  int* misc = rpre + kMaxRows + 1;  // rows, candidates, work items taken
  int* fidx = misc + 8;             // [nblk][V] where the reduced slots of each power block go
  // partial sums of the split triple terms: trs [nb][nblk][10]
  constexpr bool kTrSplit = kTrSplitOf<R, MB>;
  R* trs = reinterpret_cast<R*>(fidx + nblk * V);
  unsigned char* btab = reinterpret_cast<unsigned char*>(trs + (kTrSplit ? nb * nblk * 10 : 0));  // [256]
  signed char* cbin = reinterpret_cast<signed char*>(btab + 256);  // bin of each candidate
  Cx* accs = reinterpret_cast<Cx*>((reinterpret_cast<uintptr_t>(cbin + cap) + 15) & ~(uintptr_t)15);

  for (int b = tid; b <= nb; b += kThreads) {
    e2[b] = args.bins.e2[b]; e2f[b] = args.bins.e2f[b];
  }
  for (int k = tid; k < kWarps * 64; k += kThreads) wcnt[k] = 0;
  // the lookup table of the FP32 bin decision
  BinLookup lk;
  lk.tab = btab;
  lk.base = __float_as_uint(args.bins.e2f[0]);
  lk.shift = 0;
  while (((__float_as_uint(args.bins.e2f[nb]) - lk.base) >> lk.shift) >= 256u) ++lk.shift;
  lk.out_lo = lk.out_hi = 0.f;  // set per chunk from the rounding windows
  for (int i = tid; i < 256; i += kThreads) {
    const float v = __uint_as_float(lk.base + ((unsigned)i << lk.shift));
    int b = 0;
    while (b + 1 < nb && args.bins.e2f[b + 1] <= v) ++b;
    btab[i] = (unsigned char)b;
  }
  // Reduced slot s of power block k (slot order of the accumulation: 14 per power, then the
  // 10 triple terms) goes to the record's float index fidx[k][s] + 2b for bin b (every array
  // of the record is [multipole][bin]); <= -2: triple-term slot -2 - fidx of trs; -1: nowhere
  for (int i = tid; i < nblk * V; i += kThreads) {
    const int k = i / V, slot = i % V, m0 = k * mb;
    int f = -1;
    if (slot < 14 * MB) {
      const int t = slot / 14, q = slot % 14, m = m0 + t;
      int idx = -1;
      if (t < mb) {
        switch (q >> 1) {
          case 0: if (m <= 2 * L.N - 1) idx = L.G(m, 0); break;
          case 1: if (m >= 1 && m <= 2 * L.N + 3) idx = L.G(-m, 0); break;
          case 2: if (m <= 2 * L.N - 2) idx = L.XX(m, 0); break;
          case 3: if (m >= 1 && m <= 2 * L.N + 6) idx = L.XX(-m, 0); break;
          case 4: if (m <= 2 * L.N) idx = L.W(m, 0); break;
          case 5: if (m <= 2 * L.N + 2) idx = L.XA(m, 0); break;
          default: if (m <= 2 * L.N) idx = L.WW(m, 0); break;
        }
      }
      f = idx >= 0 ? 2 * idx + (slot & 1) : -1;
    } else if (slot < 14 * MB + 10) {
      if (kTrSplit) f = -2 - (slot - 14 * MB);
      else f = m0 == 0 ? 2 * L.TR((slot - 14 * MB) >> 1, 0) + (slot & 1) : -1;
    }
    fidx[i] = f;
  }
  // the reduced slots this lane holds after the transposed butterfly: base + [0, V/32)
  const int rbase = (lane & 16 ? V / 2 : 0) + (lane & 8 ? V / 4 : 0) + (lane & 4 ? V / 8 : 0) +
                    (lane & 2 ? V / 16 : 0) + (lane & 1 ? V / 32 : 0);
  const double rmax = args.bins.rmax * (1.0 + 1e-9) + 1e-12;
  double cell_w = -1.0;  // cell side the rounding windows were computed for

  for (int c = blockIdx.x; c < args.plan.total; c += gridDim.x) {
    // the record's segment: its catalogue's grid and centre (padding records are skipped)
    int j = 0;
    const int si = seg_of(args.plan, c, &j);
    if (si < 0 || j >= seg_live(args.plan.seg[si])) continue;  // uniform over the block
    const WaveSeg& sg = args.plan.seg[si];
    const GridGeom gm = *sg.geom;
    const double gx0 = gm.x0, gy0 = gm.y0, cell = gm.cell;
    const int gncx = gm.ncx, gncy = gm.ncy;
    if (cell != cell_w) {
      __syncthreads();
      for (int b = tid; b <= nb; b += kThreads) {
        // rounding window of the float bin decision: |dx| carries ~2 ulp of max(cell, r)
        const double e = sqrt(args.bins.e2[b]);
        const double err = 4.0 * 1.2e-7 * (cell + e);
        win[b] = (float)(2.0 * e * err + err * err);
      }
      cell_w = cell;
    }
    const int pi = sg.centres[sg.w0 + j];
    const double pxi = args.cen.px[pi], pyi = args.cen.py[pi];
    // the centre in the neighbours' grid frame: cell corner and offset as float, by the
    // arithmetic that builds the neighbours' (cell corner, offset) pairs
    float4 Pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sizeof(R) == 4) {
      const int ccx = min(max((int)floor((pxi - gx0) * gm.inv_cell), 0), gncx - 1);
      const int ccy = min(max((int)floor((pyi - gy0) * gm.inv_cell), 0), gncy - 1);
      Pi = make_float4((float)ccx * gm.cellf, (float)ccy * gm.cellf, (float)((pxi - gx0) - (double)ccx * cell),
                       (float)((pyi - gy0) - (double)ccy * cell));
    }
    if (warp == 0) {
      // the rows of cells within rmax of the centre, one per lane (cells are at least rmax / 16
      // wide, so there are at most 34), kept in row order when they hold galaxies
      const double xc = pxi - gx0, yc = pyi - gy0;
      const int cy0 = max((int)floor((yc - rmax) / cell), 0);
      const int cy1 = min((int)floor((yc + rmax) / cell), gncy - 1);
      int nr = 0, tot = 0;
      for (int cyb = cy0; cyb <= cy1; cyb += 32) {
        const int cy = cyb + lane;
        int a = 0, len = 0;
        if (cy <= cy1) {
          const double lo = cy * cell, hi = lo + cell;
          const double gap = fmax(0.0, fmax(lo - yc, yc - hi));
          if (gap <= rmax) {
            const double hw = sqrt(fmax(0.0, rmax * rmax - gap * gap));
            const int cx0 = max((int)floor((xc - hw) / cell), 0);
            const int cx1 = min((int)floor((xc + hw) / cell), gncx - 1);
            if (cx0 <= cx1) {
              a = sg.cell_start[cy * gncx + cx0];
              len = max(sg.cell_start[cy * gncx + cx1 + 1] - a, 0);
            }
          }
        }
        const unsigned ok = __ballot_sync(kFull, len > 0);
        const int pos = nr + __popc(ok & ((1u << lane) - 1u));
        const bool keep = len > 0 && pos < kMaxRows;
        int inc = keep ? len : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(kFull, inc, o);
          if (lane >= o) inc += v;
        }
        if (keep) {
          rstart[pos] = a;
          rpre[pos] = tot + inc - len;
        }
        nr = min(nr + __popc(ok), kMaxRows);
        tot += __shfl_sync(kFull, inc, 31);
      }
      if (lane == 0) {
        rpre[nr] = tot;
        misc[0] = nr; misc[1] = tot;
      }
    }
    // the record collects in shared memory
    Cx* dst = rec + (size_t)c * L.rec;
    R* accf = reinterpret_cast<R*>(accs);
    for (int k = tid; k < L.rec; k += kThreads) accs[k] = cmk<Cx>(R(0), R(0));
    if (kTrSplit)
      for (int i = tid; i < nb * nblk * 10; i += kThreads) trs[i] = R(0);
    __syncthreads();
    const int nr = misc[0], total = misc[1];
    unsigned long long pairs_here = 0;

    for (int cpos = 0; cpos < total;) {
      // ---- classification and stable bucketing by bin of the next cap candidates
      const int cend = min(total, cpos + cap);
      if (tid == 0) misc[2] = 0;  // work items of this chunk taken so far (read after the barriers below)
      bucket_chunk<R, kWarps>(cat, rstart, rpre, nr, cpos, cend, pxi, pyi, Pi, e2, e2f, win, lk, nb, cbin, wcnt, off,
                              [&](int dst, R ur, R ui, int q) {
                                R xr, xi, ww, vr, vi;
                                Pair<R>::load_x(cat, q, xr, xi, ww);
                                cpow5<R>(ur, ui, mb, vr, vi);
                                V4 e;
                                e.x = ur; e.y = ui; e.z = vr; e.w = vi;
                                euv[dst] = e;
                                ex[dst] = cmk<Cx>(xr, xi);
                                ew[dst] = ww;
                              });
      // ---- pass 3: the work items (bin, power block) of the chunk, outer bins (the fuller
      // ones) first, each taken by the next free warp; an item's sums go straight into the
      // record, whose entries no other item of the chunk touches
      const int nitems = nb * nblk;
      int item = 0;
      if (lane == 0) item = atomicAdd(&misc[2], 1);
      item = __shfl_sync(kFull, item, 0);
      while (item < nitems) {
        // the warp's next item is requested now and used at the end of this one
        int next = 0;
        if (lane == 0) next = atomicAdd(&misc[2], 1);
        const int b = nb - 1 - item / nblk, k = item % nblk, m0 = k * mb;
        const int s0 = off[b], s1 = off[b + 1];
        if (s0 < s1) {
          R a[V];
#pragma unroll
          for (int j = 0; j < V; ++j) a[j] = R(0);
          // two pairs per lane and iteration: two independent power recurrences
          auto accumulate = [&](int e0, int e1) {
            if constexpr (sizeof(R) == 4) return;  // the FP32 path runs accumulate_f32x2
            const bool two = e1 < s1;
            const int e1c = two ? e1 : e0;
            const V4 q0 = euv[e0], q1 = euv[e1c];
            const Cx xx0 = ex[e0], xx1 = ex[e1c];
            const R ur0 = q0.x, ui0 = q0.y, vr0 = q0.z, vi0 = q0.w;
            const R ur1 = q1.x, ui1 = q1.y, vr1 = q1.z, vi1 = q1.w;
            const R xr0 = xx0.x, xi0 = xx0.y, w0 = ew[e0];
            // the second pair adds nothing when it is absent
            const R xr1 = two ? xx1.x : R(0), xi1 = two ? xx1.y : R(0), w1 = two ? ew[e1c] : R(0);
            R pr0, pi0, pr1, pi1;
            cpow5<R>(vr0, vi0, k, pr0, pi0);
            cpow5<R>(vr1, vi1, k, pr1, pi1);
            const R x2r0 = xr0 * xr0 - xi0 * xi0, x2i0 = R(2) * xr0 * xi0, xa0 = xr0 * xr0 + xi0 * xi0;
            const R x2r1 = xr1 * xr1 - xi1 * xi1, x2i1 = R(2) * xr1 * xi1, xa1 = xr1 * xr1 + xi1 * xi1;
            const R ww0 = w0 * w0, ww1 = w1 * w1;
            // one power at a time; every slot is updated by two separate multiply-adds
            // (a sum of products would cost a multiply, a fused multiply-add and an add)
            auto step = [&](int t) {
              a[14 * t + 0] += xr0 * pr0;   a[14 * t + 0] += xr1 * pr1;
              a[14 * t + 1] += xr0 * pi0;   a[14 * t + 1] += xr1 * pi1;
              a[14 * t + 2] += xi0 * pr0;   a[14 * t + 2] += xi1 * pr1;
              a[14 * t + 3] += xi0 * pi0;   a[14 * t + 3] += xi1 * pi1;
              a[14 * t + 4] += x2r0 * pr0;  a[14 * t + 4] += x2r1 * pr1;
              a[14 * t + 5] += x2r0 * pi0;  a[14 * t + 5] += x2r1 * pi1;
              a[14 * t + 6] += x2i0 * pr0;  a[14 * t + 6] += x2i1 * pr1;
              a[14 * t + 7] += x2i0 * pi0;  a[14 * t + 7] += x2i1 * pi1;
              a[14 * t + 8] += w0 * pr0;    a[14 * t + 8] += w1 * pr1;
              a[14 * t + 9] += w0 * pi0;    a[14 * t + 9] += w1 * pi1;
              a[14 * t + 10] += xa0 * pr0;  a[14 * t + 10] += xa1 * pr1;
              a[14 * t + 11] += xa0 * pi0;  a[14 * t + 11] += xa1 * pi1;
              a[14 * t + 12] += ww0 * pr0;  a[14 * t + 12] += ww1 * pr1;
              a[14 * t + 13] += ww0 * pi0;  a[14 * t + 13] += ww1 * pi1;
              const R n0 = pr0 * ur0 - pi0 * ui0;
              pi0 = pr0 * ui0 + pi0 * ur0;
              pr0 = n0;
              const R n1 = pr1 * ur1 - pi1 * ui1;
              pi1 = pr1 * ui1 + pi1 * ur1;
              pr1 = n1;
            };
            if (mb == MB) {  // the common case: a full block, no predicates
#pragma unroll
              for (int t = 0; t < MB; ++t) step(t);
            } else {
#pragma unroll
              for (int t = 0; t < MB; ++t)
                if (t < mb) step(t);
            }
            if (m0 == 0) {
              // x^3 u^-8, x^3 u^-4, x^2 x^* u^-4, x^2 x^*, w^3 (the second pair is zero if absent)
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const R ur = q ? ur1 : ur0, ui = q ? ui1 : ui0, xr = q ? xr1 : xr0, xi = q ? xi1 : xi0;
                const R x2r = q ? x2r1 : x2r0, x2i = q ? x2i1 : x2i0, xa = q ? xa1 : xa0;
                const R ww = q ? w1 : w0, w2 = q ? ww1 : ww0;
                R u2r = ur * ur - ui * ui, u2i = R(2) * ur * ui;
                R u4r = u2r * u2r - u2i * u2i, u4i = R(2) * u2r * u2i;
                R u8r = u4r * u4r - u4i * u4i, u8i = R(2) * u4r * u4i;
                R x3r = x2r * xr - x2i * xi, x3i = x2r * xi + x2i * xr;
                R xcr = xa * xr, xci = xa * xi;  // x^2 x^* = |x|^2 x
                constexpr int o = 14 * MB;
                a[o + 0] += x3r * u8r + x3i * u8i;  // x3 * conj(u8)
                a[o + 1] += x3i * u8r - x3r * u8i;
                a[o + 2] += x3r * u4r + x3i * u4i;
                a[o + 3] += x3i * u4r - x3r * u4i;
                a[o + 4] += xcr * u4r + xci * u4i;
                a[o + 5] += xci * u4r - xcr * u4i;
                a[o + 6] += xcr;
                a[o + 7] += xci;
                a[o + 8] += w2 * ww;
              }
            }
          };
          if constexpr (kTrSplit)
            accumulate1_f32x2<MB>(reinterpret_cast<float*>(a), reinterpret_cast<const float4*>(euv),
                                  reinterpret_cast<const float2*>(ex), reinterpret_cast<const float*>(ew), s0,
                                  s1, lane, k, mb, args.nblk);
          else if constexpr (sizeof(R) == 4)
            accumulate_f32x2<MB>(reinterpret_cast<float*>(a), reinterpret_cast<const float4*>(euv),
                                 reinterpret_cast<const float2*>(ex), reinterpret_cast<const float*>(ew), s0,
                                 s1, lane, k, mb, m0 == 0);
          else
            for (int e = s0 + lane; e < s1; e += 64) accumulate(e, e + 32);
          // the item's record entries (their current values load while the lanes reduce)
          int f[V / 32];
          R cur[V / 32];
#pragma unroll
          for (int j = 0; j < V / 32; ++j) {
            f[j] = fidx[k * V + rbase + j];
            cur[j] = f[j] >= 0 ? accf[f[j] + 2 * b] : R(0);
          }
          // with R = sum Re(x) u^m = (a0, a1) and I = sum Im(x) u^m = (a2, a3):
          //   sum x u^m = (a0 - a3, a1 + a2),  sum x conj(u^m) = (a0 + a3, a2 - a1)
#pragma unroll
          for (int t = 0; t < MB; ++t) {
#pragma unroll
            for (int q = 0; q < 8; q += 4) {
              const R r0 = a[14 * t + q], r1 = a[14 * t + q + 1], i0 = a[14 * t + q + 2], i1 = a[14 * t + q + 3];
              a[14 * t + q] = r0 - i1;
              a[14 * t + q + 1] = r1 + i0;
              a[14 * t + q + 2] = r0 + i1;
              a[14 * t + q + 3] = i0 - r1;
            }
          }
          reduce_transpose<R, V>(a, lane);
#pragma unroll
          for (int j = 0; j < V / 32; ++j) {
            if (f[j] >= 0) accf[f[j] + 2 * b] = cur[j] + a[j];
            else if (kTrSplit && f[j] <= -2) trs[(b * nblk + k) * 10 + (-2 - f[j])] += a[j];
          }
        }
        item = __shfl_sync(kFull, next, 0);
      }
      pairs_here += (unsigned long long)off[nb];
      cpos = cend;
      __syncthreads();
    }
    if (kTrSplit) {
      // triple terms: the power blocks' sums, in block order
      for (int i = tid; i < nb * 10; i += kThreads) {
        const int b = i / 10, q = i % 10;
        R sum = R(0);
        for (int k = 0; k < nblk; ++k) sum += trs[(b * nblk + k) * 10 + q];
        accf[2 * L.TR(q >> 1, b) + (q & 1)] += sum;
      }
    }
    __syncthreads();
    if (args.accumulate) {
      for (int k = tid; k < L.rec; k += kThreads) dst[k] = cadd(dst[k], accs[k]);
    } else {
      for (int k = tid; k < L.rec; k += kThreads) dst[k] = accs[k];
    }
    if (tid == 0 && !args.accumulate) {
      R xr, xi, ww;
      Pair<R>::load_x(args.cen, pi, xr, xi, ww);
      xw[2 * (size_t)c] = cmk<Cx>(xr, xi);
      xw[2 * (size_t)c + 1] = cmk<Cx>(ww, R(0));
    }
    if (tid == 0) {
      atomicAdd(args.pair_count, pairs_here);
    }
    __syncthreads();
  }
}

// powers per warp block and resident CTAs per SM: FP32 runs two CTAs of 8 warps per SM
// (3 powers per block keep the accumulators within 128 registers, and each CTA gets half
// of the shared memory), FP64 one CTA with 3 powers per block
template <typename R> constexpr int kMB = sizeof(R) == 4 ? 6 : 3;
template <typename R> constexpr int kMinBlocks = sizeof(R) == 4 ? 2 : 1;

}  // namespace

template <typename R>
cudaError_t gather_wave(const SortedCat& cat, const SortedCat& cen, const Bins& bins, const Layout& L,
                        const WavePlan& plan, bool accumulate, cplx_t<R>* rec, cplx_t<R>* xw,
                        unsigned long long* pair_count, int sm_count, cudaStream_t s) {
  if (plan.total <= 0) return cudaSuccess;
  constexpr int MB = kMB<R>;
  constexpr int MINB = kMinBlocks<R>;
  GatherArgs a;
  a.cat = cat; a.cen = cen; a.accumulate = accumulate ? 1 : 0;
  a.bins = bins; a.L = L; a.plan = plan; a.pair_count = pair_count;
  const int npow = L.max_pow + 1;
  const int nblk = (npow + MB - 1) / MB;  // the warps take (bin, block) items in turn
  a.mb = (npow + nblk - 1) / nblk;
  a.nblk = (npow + a.mb - 1) / a.mb;
  const size_t fixed = (size_t)L.rec * sizeof(cplx_t<R>) + 16 + 65 * sizeof(double) + 130 * sizeof(float) +
                       (65 + kWarps * 64 + 2 * kMaxRows + 1 + 8 + (size_t)a.nblk * GCfg<R, MB>::V) * sizeof(int) + 256 +
                       64 + (kTrSplitOf<R, MB> ? (size_t)bins.nb * a.nblk * 10 * sizeof(R) : 0);
  const size_t budget = MINB == 1 ? 227 * 1024 : 113 * 1024;
  constexpr size_t per_pair = sizeof(typename Vec4<R>::T) + sizeof(cplx_t<R>) + sizeof(R) + 1;
  if (fixed + per_pair * kThreads > budget) return cudaErrorInvalidConfiguration;
  int cap = (int)((budget - fixed) / per_pair);
  cap = cap / kThreads * kThreads;
  if (cap > 8192) cap = 8192;
  a.cap = cap;
  const size_t smem = fixed + (size_t)cap * per_pair;
  cudaError_t e = cudaFuncSetAttribute(gather_kernel<R, MB, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = plan.total;
  gather_kernel<R, MB, MINB><<<grid, kThreads, smem, s>>>(a, rec, xw);
  ++g_launches;
  (void)sm_count;
  return cudaGetLastError();
}

template cudaError_t gather_wave<float>(const SortedCat&, const SortedCat&, const Bins&, const Layout&,
                                        const WavePlan&, bool, float2*, float2*, unsigned long long*, int,
                                        cudaStream_t);
template cudaError_t gather_wave<double>(const SortedCat&, const SortedCat&, const Bins&, const Layout&,
                                         const WavePlan&, bool, double2*, double2*, unsigned long long*, int,
                                         cudaStream_t);

}  // namespace ext4pcf
