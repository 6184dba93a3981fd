// Direct estimator of <M_ap^2> and <M_ap^4> (paper Sect. 5.2, Eq. MapDirectEstimator) on the
// cell grid of the catalogue.
//
// Per aperture (centre vartheta, radius theta) the distinct quadruplet sums of
// a_i = w_i Q_theta(|vartheta_i - vartheta|) gamma_t,i and of w_i are 4! times the elementary
// symmetric polynomials e_4(a), e_4(w), which follow from the power sums p_k = sum_i a_i^k
// (k = 1..4) by Newton's identities; that makes the estimator linear in the galaxies of
// the aperture (the accelerated form the paper uses).  Galaxies enter when
// |vartheta_i - vartheta| < 4 theta (the hard cut of the filter support).
//
// With u = dx / theta, v = dy / theta, Eq. CrittendenQ and Eq. gammatx_def combine into
//   a_i = -(w gamma_1 (u^2 - v^2) + 2 w gamma_2 u v) exp(-(u^2 + v^2) / 2) / (4 pi theta^2),
// the factor 1 / r^2 of cos 2 zeta and sin 2 zeta cancelling the r^2 of the filter.
//
// Kernels (one launch of each per radius):
//   aperture_prep    one thread per aperture: the cell of the centre and its offset inside the
//                    cell (FP64 once per aperture; the kernels below use no FP64 on their
//                    per-galaxy path);
//   aperture_sums    one WARP per (aperture, row split): scans the cell rows that meet the disc
//                    (each row a contiguous range of the cell-sorted catalogue), evaluates a_i
//                    in FP32 and accumulates the eight power sums of a and w, in FP32 over at
//                    most 32 galaxies per lane and then into unevaluated FP32 pairs (hi + lo,
//                    error-free two-sum), reduced across the warp the same way;
//   aperture_finish  one thread per aperture: adds the splits in order in FP64, applies
//                    Newton's identities and writes the aperture record; one partial sum of
//                    the records per block;
//   aperture_moments one CTA: adds the block partials in order into the per-radius sums and
//                    derives <M_ap^4>, <M_ap^2> and the connected part.
//
// Row and chord limits are computed in FP32 in cell units relative to the aperture's cell:
// every bound is widened by a slack (1e-3 cell, above the FP32 rounding of quantities up to
// the largest cut radius of 4096 cells) and the squared half-chord by a bound on its rounding
// error, so every galaxy inside the cut lies in a scanned cell; scanning a few extra cells is
// harmless (the cut decides).  Cut decisions: the FP32 distance is exact enough (relative
// error < 1e-6) that galaxies further than a relative 1e-5 from the cut radius are classified
// correctly in FP32; those inside that band are decided again in FP64 as
// (x - x_c)^2 + (y - y_c)^2 < (4 theta)^2 with separately rounded products.
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"

namespace ext4pcf {
namespace {

constexpr int kApThreads = 128;
constexpr int kApWarps = kApThreads / 32;
constexpr int kWarpRows = 256;  // rows per chunk of one warp
constexpr int kPromote = 32;    // galaxies per lane between FP32 partial flushes
constexpr float kSlack = 1e-3f; // cell units
constexpr int kSumFloats = 20;  // per work item: 8 (hi, lo) pairs, count, padding

struct ApArgs {
  const float4* p4;
  const float4* s4;
  const double* px;
  const double* py;
  const int* cell_start;
  int ncx, ncy;
  float cellf;
  float rc;               // cut radius 4 theta in cells (float)
  float invt;             // 1 / theta
  const double* centres;  // [n_ap][2]
  const int4* prep;       // [n_ap]: cell x, cell y, offset x, offset y (cells, float bits)
  int nsplit;
  long long n_items;      // n_ap * nsplit
  double R2;              // (4 theta)^2
  float* sums;            // [n_items][kSumFloats]
};

__global__ void aperture_prep(const double* __restrict__ centres, int n_ap, double x0, double y0, double cell,
                              double inv_cell, int ncx, int ncy, double R, int4* __restrict__ prep) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_ap) return;
  const double ax = centres[2 * a], ay = centres[2 * a + 1];
  // a disc that cannot reach the grid (or a non-finite centre) holds no galaxy: marked empty,
  // so that the cell indices below stay within a few thousand of the grid
  const double mx = R + 2.0 * cell;
  if (!(ax >= x0 - mx && ax <= x0 + ncx * cell + mx && ay >= y0 - mx && ay <= y0 + ncy * cell + mx)) {
    prep[a] = make_int4(INT_MIN, 0, 0, 0);
    return;
  }
  const double cx = floor((ax - x0) * inv_cell), cy = floor((ay - y0) * inv_cell);
  const float ox = (float)(((ax - x0) - cx * cell) * inv_cell);
  const float oy = (float)(((ay - y0) - cy * cell) * inv_cell);
  prep[a] = make_int4((int)cx, (int)cy, __float_as_int(ox), __float_as_int(oy));
}

// (hi, lo) += b with the rounding error of hi + b kept in lo (two-sum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (b - bb);
  hi = s;
}

__global__ void __launch_bounds__(kApThreads) aperture_sums(ApArgs A) {
  __shared__ int s_start[kApWarps][kWarpRows];
  __shared__ int s_pre[kApWarps][kWarpRows + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long item = (long long)blockIdx.x * kApWarps + wid;
  if (item >= A.n_items) return;  // whole warp; no block-level barrier below
  const int ap = (int)(item / A.nsplit), sp = (int)(item % A.nsplit);
  const int4 pr = A.prep[ap];
  float H[8] = {0, 0, 0, 0, 0, 0, 0, 0}, L[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cnt = 0;
  if (pr.x != INT_MIN) {
    const int acx = pr.x, acy = pr.y;
    const float ox = __int_as_float(pr.z), oy = __int_as_float(pr.w);
    const float Rs = A.rc + kSlack;
    const float h2err = 1e-6f * (A.rc + 2.f) * (A.rc + 2.f);
    const int ylo = max(acy + (int)floorf(oy - Rs), 0);
    const int yhi = min(acy + (int)floorf(oy + Rs), A.ncy - 1);
    if (ylo <= yhi) {
      const int nrow = yhi - ylo + 1;
      const int ra = ylo + (int)((long long)nrow * sp / A.nsplit);
      const int rz = ylo + (int)((long long)nrow * (sp + 1) / A.nsplit);  // exclusive
      // float distance: (corner_j - corner_c) is exact (power-of-two cell), offsets are small
      const float acxf = (float)acx * A.cellf, acyf = (float)acy * A.cellf;
      const float fxf = ox * A.cellf, fyf = oy * A.cellf;
      const float invt = A.invt;
      const float band = 16.f * 1e-5f * (1.f + A.cellf * invt);
      for (int r0 = ra; r0 < rz; r0 += kWarpRows) {
        const int nr = min(kWarpRows, rz - r0);
        const int per = (nr + 31) >> 5;
        const int rb = min(lane * per, nr), re = min(rb + per, nr);
        int mine = 0;
        for (int r = rb; r < re; ++r) {
          const int cy = r0 + r;
          const float k = (float)(cy - acy);
          const float dymin = fmaxf(0.f, fmaxf(k - oy, oy - (k + 1.f)));
          int b = 0, len = 0;
          if (dymin < Rs) {
            const float h = sqrtf(fmaf(Rs, Rs, -dymin * dymin) + h2err) + kSlack;
            const int xl = max(acx + (int)floorf(ox - h), 0);
            const int xh = min(acx + (int)floorf(ox + h), A.ncx - 1);
            if (xl <= xh) {
              const int row = cy * A.ncx;
              b = A.cell_start[row + xl];
              len = A.cell_start[row + xh + 1] - b;
            }
          }
          s_start[wid][r] = b;
          s_pre[wid][r] = len;
          mine += len;
        }
        // exclusive scan of the per-lane galaxy counts over the warp
        int incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int run = incl - mine;
        for (int r = rb; r < re; ++r) {
          const int len = s_pre[wid][r];
          s_pre[wid][r] = run;
          run += len;
        }
        if (lane == 0) s_pre[wid][nr] = total;
        __syncwarp();
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int kk = 0, r = 0;
        for (int v = lane; v < total; v += 32) {
          while (s_pre[wid][r + 1] <= v) ++r;
          const int j = s_start[wid][r] + (v - s_pre[wid][r]);
          const float4 p = A.p4[j];
          const float4 g = A.s4[j];
          const float dx = (p.x - acxf) + (p.z - fxf);
          const float dy = (p.y - acyf) + (p.w - fyf);
          const float u = dx * invt, w = dy * invt;
          const float r2n = fmaf(u, u, w * w);
          bool in = r2n < 16.f;
          if (fabsf(r2n - 16.f) <= band) {
            const double ddx = A.px[j] - A.centres[2 * ap], ddy = A.py[j] - A.centres[2 * ap + 1];
            in = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)) < A.R2;
          }
          if (in) {
            const float e = expf(-0.5f * r2n);
            const float b = -e * fmaf(g.x, fmaf(u, u, -w * w), 2.f * g.y * u * w);
            const float b2 = b * b, w2 = g.z * g.z;
            f[0] += b; f[1] += b2; f[2] += b2 * b; f[3] += b2 * b2;
            f[4] += g.z; f[5] += w2; f[6] += w2 * g.z; f[7] += w2 * w2;
            ++cnt;
          }
          if (++kk == kPromote) {
#pragma unroll
            for (int i = 0; i < 8; ++i) { two_sum_acc(H[i], L[i], f[i]); f[i] = 0.f; }
            kk = 0;
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) two_sum_acc(H[i], L[i], f[i]);
        __syncwarp();  // s_start / s_pre are rewritten by the next chunk
      }
    }
  }
  // warp reduction of the (hi, lo) pairs and the count
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float h2 = __shfl_xor_sync(0xffffffffu, H[i], o);
      const float l2 = __shfl_xor_sync(0xffffffffu, L[i], o);
      two_sum_acc(H[i], L[i], h2);
      L[i] += l2;
    }
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (lane == 0) {
    float4* o = reinterpret_cast<float4*>(A.sums + item * kSumFloats);
    o[0] = make_float4(H[0], L[0], H[1], L[1]);
    o[1] = make_float4(H[2], L[2], H[3], L[3]);
    o[2] = make_float4(H[4], L[4], H[5], L[5]);
    o[3] = make_float4(H[6], L[6], H[7], L[7]);
    o[4] = make_float4(__int_as_float(cnt), 0.f, 0.f, 0.f);
  }
}

// e_1, e_2, e_4 from the power sums p_1..p_4 (Newton's identities)
__device__ __forceinline__ void newton(const double p[5], double n, double& e1, double& e2, double& e4) {
  e1 = p[1];
  e2 = (e1 * p[1] - p[2]) * 0.5;
  const double e3 = (e2 * p[1] - e1 * p[2] + p[3]) / 3.0;
  e4 = (e3 * p[1] - e2 * p[2] + e1 * p[3] - p[4]) * 0.25;
  // fewer galaxies than the order: the distinct sum is empty (exactly zero)
  if (n < 2.0) e2 = 0.0;
  if (n < 4.0) e4 = 0.0;
  if (n < 1.0) e1 = 0.0;
}

constexpr int kFinThreads = 128;

__global__ void __launch_bounds__(kFinThreads) aperture_finish(const float* __restrict__ sums, int n_ap, int nsplit,
                                                               double theta, double* __restrict__ rec,
                                                               double* __restrict__ part) {
  __shared__ double red[4][kFinThreads];
  const int ap = blockIdx.x * kFinThreads + threadIdx.x;
  double t[4] = {0, 0, 0, 0};
  if (ap < n_ap) {
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long n = 0;
    for (int sp = 0; sp < nsplit; ++sp) {
      const float4* q = reinterpret_cast<const float4*>(sums + ((long long)ap * nsplit + sp) * kSumFloats);
      for (int i = 0; i < 4; ++i) {
        const float4 v = q[i];
        s[2 * i] += (double)v.x + (double)v.y;
        s[2 * i + 1] += (double)v.z + (double)v.w;
      }
      n += __float_as_int(q[4].x);
    }
    const double c = 1.0 / (4.0 * M_PI * theta * theta);  // a = b c
    const double pa[5] = {0.0, s[0] * c, s[1] * c * c, s[2] * c * c * c, s[3] * (c * c) * (c * c)};
    const double pw[5] = {0.0, s[4], s[5], s[6], s[7]};
    const double nn = (double)n;
    double a1, a2, a4, w1, w2, w4;
    newton(pa, nn, a1, a2, a4);
    newton(pw, nn, w1, w2, w4);
    double* o = rec + (size_t)ap * 8;
    o[0] = a1; o[1] = a2; o[2] = a4; o[3] = w1; o[4] = w2; o[5] = w4; o[6] = nn; o[7] = 0.0;
    t[0] = a4; t[1] = w4; t[2] = a2; t[3] = w2;
  }
  for (int i = 0; i < 4; ++i) red[i][threadIdx.x] = t[i];
  __syncthreads();
  for (int st = kFinThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int i = 0; i < 4; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[(size_t)blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

constexpr int kMomThreads = 256;

__global__ void __launch_bounds__(kMomThreads) aperture_moments(const double* __restrict__ part, int nblk, int n_ap,
                                                               double theta, double* __restrict__ mom) {
  __shared__ double red[4][kMomThreads];
  double t[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += kMomThreads)
    for (int i = 0; i < 4; ++i) t[i] += part[(size_t)b * 4 + i];
  for (int i = 0; i < 4; ++i) red[i][threadIdx.x] = t[i];
  __syncthreads();
  for (int st = kMomThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int i = 0; i < 4; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mom[i] += red[i][0];
    mom[4] += (double)n_ap;
    const double area = M_PI * (4.0 * theta) * (4.0 * theta);
    const double a2 = area * area;
    mom[5] = mom[1] > 0.0 ? a2 * a2 * mom[0] / mom[1] : 0.0;
    mom[6] = mom[3] > 0.0 ? a2 * mom[2] / mom[3] : 0.0;
    mom[7] = mom[5] - 3.0 * mom[6] * mom[6];
  }
}

}  // namespace

int map_direct_splits(int n_ap, int sm_count, double theta, double cell) {
  // enough warps for several waves of the GPU, never more splits than about one per 4 rows
  const int rows = (int)std::min(1.0e6, 8.0 * theta / cell) + 2;
  int ns = (32 * sm_count + n_ap - 1) / std::max(n_ap, 1);
  ns = std::max(1, std::min(ns, std::max(1, rows / 4)));
  while (ns > 1 && (long long)ns * n_ap > (1LL << 34)) --ns;
  return ns;
}

size_t map_direct_scratch(int n_ap, int nsplit) {
  const size_t nblk = (size_t)(n_ap + kFinThreads - 1) / kFinThreads;
  return (size_t)n_ap * 16 + (size_t)n_ap * nsplit * kSumFloats * 4 + nblk * 32 + 256;
}

cudaError_t map_direct_radius(const SortedCat& cat, const double* centres, int n_ap, double theta,
                              int nsplit, void* scratch, double* rec, double* mom, cudaStream_t s) {
  const int nblk = (n_ap + kFinThreads - 1) / kFinThreads;
  int4* prep = (int4*)scratch;
  float* sums = (float*)((char*)scratch + (size_t)n_ap * 16);
  double* part = (double*)((char*)sums + (((size_t)n_ap * nsplit * kSumFloats * 4 + 255) / 256) * 256);
  const long long n_items = (long long)n_ap * nsplit;
  if (n_ap > 0) {
    if (cat.n > 0) {
      aperture_prep<<<(n_ap + 127) / 128, 128, 0, s>>>(centres, n_ap, cat.x0, cat.y0, cat.cell, 1.0 / cat.cell,
                                                        cat.ncx, cat.ncy, 4.0 * theta, prep);
      ApArgs A;
      A.p4 = cat.p4; A.s4 = cat.s4; A.px = cat.px; A.py = cat.py; A.cell_start = cat.cell_start;
      A.ncx = cat.ncx; A.ncy = cat.ncy; A.cellf = cat.cellf;
      A.rc = (float)(4.0 * theta / cat.cell);
      A.invt = (float)(1.0 / theta);
      A.centres = centres; A.prep = prep; A.nsplit = nsplit; A.n_items = n_items;
      const double R = 4.0 * theta;
      A.R2 = R * R;  // the oracle's (4 theta)^2, one rounding
      A.sums = sums;
      aperture_sums<<<(unsigned)((n_items + kApWarps - 1) / kApWarps), kApThreads, 0, s>>>(A);
      g_launches += 2;
    } else {
      cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)n_items * kSumFloats * 4, s);
      if (e != cudaSuccess) return e;
    }
    aperture_finish<<<nblk, kFinThreads, 0, s>>>(sums, n_ap, nsplit, theta, rec, part);
    ++g_launches;
  }
  aperture_moments<<<1, kMomThreads, 0, s>>>(part, nblk, n_ap, theta, mom);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ext4pcf
