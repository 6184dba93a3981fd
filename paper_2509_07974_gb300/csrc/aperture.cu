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
//   aperture_sums    one CTA per (aperture, row split): scans the cell rows that meet the disc
//                    (each row is one contiguous range of the cell-sorted catalogue), evaluates
//                    a_i in FP32 and accumulates the eight power sums of a and w in FP32 over
//                    at most 32 galaxies per thread before promoting them to FP64;
//   aperture_finish  one thread per aperture: adds the splits in order, applies Newton's
//                    identities in FP64 and writes the aperture record;
//   aperture_moments one CTA: adds the records of all apertures (fixed order) into the
//                    per-radius sums and derives <M_ap^4>, <M_ap^2> and the connected part.
//
// Cut decisions: the FP32 distance is exact enough (relative error < 1e-6) that galaxies
// further than a relative 1e-5 from the cut radius are classified correctly in FP32; those
// inside that band are decided again in FP64 as (x - x_c)^2 + (y - y_c)^2 < (4 theta)^2
// with separately rounded products.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace ext4pcf {
namespace {

constexpr int kApThreads = 128;
constexpr int kApWarps = kApThreads / 32;
constexpr int kRowsChunk = 1024;
constexpr int kPromote = 32;

struct ApArgs {
  const float4* p4;
  const float4* s4;
  const double* px;
  const double* py;
  const int* cell_start;
  int ncx, ncy;
  double x0, y0, cell, inv_cell;
  float cellf;
  const double* centres;  // [n_ap][2]
  int n_ap, nsplit;
  double theta;
  double* sums;  // [n_ap][nsplit][9]: power sums of a/c (k = 1..4), of w (k = 1..4), count
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kApThreads) aperture_sums(ApArgs A) {
  __shared__ int s_start[kRowsChunk];
  __shared__ int s_pre[kRowsChunk + 1];
  __shared__ int s_tot[kApWarps];
  __shared__ double s_red[kApWarps][9];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ap = blockIdx.x / A.nsplit, sp = blockIdx.x % A.nsplit;
  const double ax = A.centres[2 * ap], ay = A.centres[2 * ap + 1];
  double P[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cnt = 0;
  if (isfinite(ax) && isfinite(ay)) {
    const double theta = A.theta, R = 4.0 * theta, R2 = __dmul_rn(R, R);
    // slack in position units that covers the rounding of cell indices and of the chord
    const double sl = A.cell * 1e-6 +
                      1e-14 * (fabs(ax) + fabs(ay) + fabs(A.x0) + fabs(A.y0) + (A.ncx + A.ncy) * A.cell);
    const double Rs = R + sl;
    double ylo = floor((ay - Rs - A.y0) * A.inv_cell), yhi = floor((ay + Rs - A.y0) * A.inv_cell);
    ylo = fmax(ylo, 0.0);
    yhi = fmin(yhi, (double)(A.ncy - 1));
    if (ylo <= yhi) {
      // this split's rows
      const long long nrow = (long long)(yhi - ylo) + 1;
      const int ra = (int)ylo + (int)(nrow * sp / A.nsplit);
      const int rz = (int)ylo + (int)(nrow * (sp + 1) / A.nsplit);  // exclusive
      // aperture cell corner (exact multiple of the power-of-two cell) and offset
      const double acx = fmin(fmax(floor((ax - A.x0) * A.inv_cell), -1048576.0), 1048576.0);
      const double acy = fmin(fmax(floor((ay - A.y0) * A.inv_cell), -1048576.0), 1048576.0);
      const float acxf = (float)acx * A.cellf, acyf = (float)acy * A.cellf;
      const float fxf = (float)((ax - A.x0) - acx * A.cell);
      const float fyf = (float)((ay - A.y0) - acy * A.cell);
      const float invt = (float)(1.0 / theta);
      const float band = 16.f * 1e-5f * (1.f + A.cellf * invt);
      for (int r0 = ra; r0 < rz; r0 += kRowsChunk) {
        const int nr = min(kRowsChunk, rz - r0);
        const int per = (nr + kApThreads - 1) / kApThreads;
        const int rb = min(tid * per, nr), re = min(rb + per, nr);
        int mine = 0;
        for (int r = rb; r < re; ++r) {
          const int cy = r0 + r;
          const double ylow = A.y0 + cy * A.cell, yhigh = ylow + A.cell;
          const double dymin = fmax(0.0, fmax(ylow - ay, ay - yhigh));
          int b = 0, len = 0;
          if (dymin < Rs) {
            const double h = sqrt(Rs * Rs - dymin * dymin);
            double xl = floor((ax - h - A.x0) * A.inv_cell), xh = floor((ax + h - A.x0) * A.inv_cell);
            xl = fmax(xl, 0.0);
            xh = fmin(xh, (double)(A.ncx - 1));
            if (xl <= xh) {
              const int row = cy * A.ncx;
              b = A.cell_start[row + (int)xl];
              len = A.cell_start[row + (int)xh + 1] - b;
            }
          }
          s_start[r] = b;
          s_pre[r] = len;
          mine += len;
        }
        // block-wide exclusive scan of the per-thread galaxy counts
        int incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) s_tot[wid] = incl;
        __syncthreads();
        int run = incl - mine, total = 0;
        for (int q = 0; q < kApWarps; ++q) {
          if (q < wid) run += s_tot[q];
          total += s_tot[q];
        }
        for (int r = rb; r < re; ++r) {
          const int len = s_pre[r];
          s_pre[r] = run;
          run += len;
        }
        if (tid == 0) s_pre[nr] = total;
        __syncthreads();
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int k = 0, r = 0;
        for (int v = tid; v < total; v += kApThreads) {
          while (s_pre[r + 1] <= v) ++r;
          const int j = s_start[r] + (v - s_pre[r]);
          const float4 p = A.p4[j];
          const float4 g = A.s4[j];
          const float dx = (p.x - acxf) + (p.z - fxf);
          const float dy = (p.y - acyf) + (p.w - fyf);
          const float u = dx * invt, w = dy * invt;
          const float r2n = fmaf(u, u, w * w);
          bool in = r2n < 16.f;
          if (fabsf(r2n - 16.f) <= band) {
            const double ddx = A.px[j] - ax, ddy = A.py[j] - ay;
            in = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)) < R2;
          }
          if (in) {
            const float e = expf(-0.5f * r2n);
            const float b = -e * fmaf(g.x, fmaf(u, u, -w * w), 2.f * g.y * u * w);
            const float b2 = b * b, w2 = g.z * g.z;
            f[0] += b; f[1] += b2; f[2] += b2 * b; f[3] += b2 * b2;
            f[4] += g.z; f[5] += w2; f[6] += w2 * g.z; f[7] += w2 * w2;
            ++cnt;
          }
          if (++k == kPromote) {
#pragma unroll
            for (int i = 0; i < 8; ++i) { P[i] += (double)f[i]; f[i] = 0.f; }
            k = 0;
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) P[i] += (double)f[i];
        __syncthreads();  // s_start / s_pre / s_tot are rewritten by the next chunk
      }
    }
  }
  // block reduction in a fixed order
  double c = warp_sum((double)cnt);
#pragma unroll
  for (int i = 0; i < 8; ++i) P[i] = warp_sum(P[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) s_red[wid][i] = P[i];
    s_red[wid][8] = c;
  }
  __syncthreads();
  if (tid < 9) {
    double t = 0;
    for (int q = 0; q < kApWarps; ++q) t += s_red[q][tid];
    A.sums[((size_t)ap * A.nsplit + sp) * 9 + tid] = t;
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

__global__ void aperture_finish(const double* __restrict__ sums, int n_ap, int nsplit, double theta,
                                double* __restrict__ rec) {
  const int ap = blockIdx.x * blockDim.x + threadIdx.x;
  if (ap >= n_ap) return;
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int sp = 0; sp < nsplit; ++sp)
    for (int i = 0; i < 9; ++i) s[i] += sums[((size_t)ap * nsplit + sp) * 9 + i];
  const double c = 1.0 / (4.0 * M_PI * theta * theta);  // a = b c
  const double pa[5] = {0.0, s[0] * c, s[1] * c * c, s[2] * c * c * c, s[3] * (c * c) * (c * c)};
  const double pw[5] = {0.0, s[4], s[5], s[6], s[7]};
  double a1, a2, a4, w1, w2, w4;
  newton(pa, s[8], a1, a2, a4);
  newton(pw, s[8], w1, w2, w4);
  double* o = rec + (size_t)ap * 8;
  o[0] = a1; o[1] = a2; o[2] = a4; o[3] = w1; o[4] = w2; o[5] = w4; o[6] = s[8]; o[7] = 0.0;
}

constexpr int kMomThreads = 256;

__global__ void __launch_bounds__(kMomThreads) aperture_moments(const double* __restrict__ rec, int n_ap,
                                                               double theta, double* __restrict__ mom) {
  __shared__ double red[4][kMomThreads];
  double t[4] = {0, 0, 0, 0};
  for (int a = threadIdx.x; a < n_ap; a += kMomThreads) {
    const double* r = rec + (size_t)a * 8;
    t[0] += r[2]; t[1] += r[5]; t[2] += r[1]; t[3] += r[4];
  }
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
  // enough CTAs for a few waves of the GPU, never more splits than about one per 8 rows
  const int rows = (int)std::min(1.0e6, 8.0 * theta / cell) + 2;
  int ns = (8 * sm_count + n_ap - 1) / std::max(n_ap, 1);
  ns = std::max(1, std::min(ns, std::max(1, rows / 8)));
  while (ns > 1 && (long long)ns * n_ap > 2147483647LL) --ns;
  return ns;
}

cudaError_t map_direct_radius(const SortedCat& cat, const double* centres, int n_ap, double theta,
                              int nsplit, double* sums, double* rec, double* mom, cudaStream_t s) {
  if (n_ap > 0) {
    if (cat.n > 0) {
      ApArgs A;
      A.p4 = cat.p4; A.s4 = cat.s4; A.px = cat.px; A.py = cat.py; A.cell_start = cat.cell_start;
      A.ncx = cat.ncx; A.ncy = cat.ncy; A.x0 = cat.x0; A.y0 = cat.y0; A.cell = cat.cell;
      A.inv_cell = 1.0 / cat.cell; A.cellf = cat.cellf;
      A.centres = centres; A.n_ap = n_ap; A.nsplit = nsplit; A.theta = theta; A.sums = sums;
      aperture_sums<<<(unsigned)((long long)n_ap * nsplit), kApThreads, 0, s>>>(A);
    } else {
      cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)n_ap * nsplit * 9 * sizeof(double), s);
      if (e != cudaSuccess) return e;
    }
    aperture_finish<<<(n_ap + 127) / 128, 128, 0, s>>>(sums, n_ap, nsplit, theta, rec);
    g_launches += cat.n > 0 ? 2 : 1;
  }
  aperture_moments<<<1, kMomThreads, 0, s>>>(rec, n_ap, theta, mom);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ext4pcf
