// FP64 transforms of the multipoles:
//  * real space (paper Eq. Multipole2RealConversion): for each component and radial-bin
//    triple, the angular density (2 pi)^-2 sum_n Upsilon_n e^{i n2 phi12 + i n3 phi13} is
//    integrated over n_phi x n_phi uniform angular bins, as a separable two-stage sum;
//    Gamma = Upsilon / N per bin (Eq. 4PCF_quadrupletestimator);
//  * fourth-order aperture measures (Eq. 4PCF2M4) for the filter of Eq. CrittendenQ, whose
//    aperture-centre integral is done in closed form: with vt_0 = 0, vt_1 = t1,
//    vt_2 = t2 e^{i phi12}, vt_3 = t3 e^{i phi13}, d_a = vt_a - (vt_1+vt_2+vt_3)/4,
//      F_mu = 2 pi t1 t2 t3 e^{i ph_mu} (4 pi theta^4)^-4 exp(-sum|d_a|^2 / 2theta^2) J_mu,
//      J_mu = sum_p P_p R_p pi p! (theta^2/2)^{p+1},
//    P(z^*) = prod over unconjugated apertures (z^* + d_a^*)^2, R(z) = prod over conjugated
//    apertures (z + d_a)^2, ph_mu = 2 sum_a s_a zeta_a of the x-projection (s = +-1).
#include <mutex>

#include "common.cuh"

namespace ext4pcf {

namespace {

constexpr double kPi = 3.14159265358979323846;

// (1/2pi) * integral of e^{i n phi} over angular bin p of n_phi uniform bins
__global__ void angle_table(int N, int nphi, double2* E) {
  const int nn = 2 * N + 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn * nphi; k += gridDim.x * blockDim.x) {
    const int t = k / nphi, p = k % nphi, n = t - N;
    const double lo = 2.0 * kPi * p / nphi, hi = 2.0 * kPi * (p + 1) / nphi;
    double re, im;
    if (n == 0) {
      re = (hi - lo) / (2.0 * kPi);
      im = 0.0;
    } else {
      double sh, ch, sl, cl;
      sincos(n * hi, &sh, &ch);
      sincos(n * lo, &sl, &cl);
      // (e^{in hi} - e^{in lo}) / (i n) / (2 pi)
      re = (sh - sl) / (n * 2.0 * kPi);
      im = -(ch - cl) / (n * 2.0 * kPi);
    }
    E[k] = make_double2(re, im);
  }
}

// Bin counts of component mu for radial triples [tri0, tri0 + gridDim.x / ncomp).
// IS_NORM: writes real N counts to out_norm[tri][p][q]; otherwise writes
// Upsilon / N to out_gam[mu][tri][p][q] (complex, accumulated), reading norm.
template <bool IS_NORM>
__global__ void real_space_kernel(const double2* __restrict__ ups, int nb, int N, int nphi,
                                  const double2* __restrict__ E, int tri0, int ntri,
                                  const double* __restrict__ norm_in, double* __restrict__ norm_out,
                                  double2* __restrict__ gam_out, size_t gam_mu_stride) {
  extern __shared__ double2 sm[];
  const int nn = 2 * N + 1;
  const int mu = IS_NORM ? 8 : (int)(blockIdx.x / ntri);
  const int lt = (int)(blockIdx.x % ntri), tri = tri0 + lt;
  const size_t nb3 = (size_t)nb * nb * nb;
  double2* U = sm;                 // [nn][nn]
  double2* T1 = sm + nn * nn;      // [nn][nphi]
  for (int k = threadIdx.x; k < nn * nn; k += blockDim.x) {
    const int a2 = k / nn, a3 = k % nn;
    U[k] = ups[(((size_t)mu * nn + a2) * nn + a3) * nb3 + tri];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nn * nphi; k += blockDim.x) {
    const int a2 = k / nphi, q = k % nphi;
    double re = 0, im = 0;
    for (int a3 = 0; a3 < nn; ++a3) {
      const double2 u = U[a2 * nn + a3], e = E[a3 * nphi + q];
      re += u.x * e.x - u.y * e.y;
      im += u.x * e.y + u.y * e.x;
    }
    T1[k] = make_double2(re, im);
  }
  __syncthreads();
  const size_t nph2 = (size_t)nphi * nphi;
  for (int k = threadIdx.x; k < nphi * nphi; k += blockDim.x) {
    const int p = k / nphi, q = k % nphi;
    double re = 0, im = 0;
    for (int a2 = 0; a2 < nn; ++a2) {
      const double2 e = E[a2 * nphi + p], t = T1[a2 * nphi + q];
      re += e.x * t.x - e.y * t.y;
      im += e.x * t.y + e.y * t.x;
    }
    const size_t o = (size_t)lt * nph2 + k;
    if (IS_NORM) {
      norm_out[o] = re;
    } else {
      const double nv = norm_in[o];
      double2& g = gam_out[(size_t)mu * gam_mu_stride + o];
      if (nv != 0.0) { g.x += re / nv; g.y += im / nv; }
    }
  }
}

__global__ void add_arrays(double* __restrict__ dst, const double* __restrict__ src, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] += src[k];
}

struct Map4Args {
  int nb, nphi, n_ap, tri0, ntri;
  double tb[32];   // representative radius per bin
  double vol[32];  // A_b / tb
  double ap[64];
};

__constant__ signed char kBeta[8][4] = {{0, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0},
                                        {0, 0, 0, 1}, {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1}};

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// block = (triple in chunk, slice of the angular bins).  The aperture-independent part of
// F_mu (Gamma_mu times the phase and geometric factors times the coefficients P_t R_t of
// J_mu) is formed once per angular bin, kM4Bins bins at a time, and kept in shared memory;
// then the threads, one per (mu, aperture) pair, fold the tile into their sums.  Only
// t <= min(deg P, deg R) contributes: 0 for mu = 0, 2 for one conjugated aperture, 4 for two.
constexpr int kM4Bins = 16;     // angular bins per tile (kM4Bins * 8 = blockDim items)
constexpr int kM4Threads = 128;
constexpr int kM4MaxPairs = 4;  // (mu, aperture) pairs per thread: 8 * 64 / 128

__global__ void __launch_bounds__(kM4Threads) map4_kernel(const Map4Args a, const double2* __restrict__ gam,
                                                          size_t gam_mu_stride, int nsplit,
                                                          double2* __restrict__ partial) {
  __shared__ double2 coef[kM4Bins][8][5];  // Gamma_mu e^{i ph_mu} geo P_t R_t, t <= 4
  __shared__ double exs[kM4Bins][64];      // e^{-sum|d|^2 / 2 theta^2} per bin and aperture
  __shared__ double sd2s[kM4Bins];
  __shared__ double hps[64][5];            // pi t! h^{t+1} / (4 pi theta^4)^4
  const size_t nph2 = (size_t)a.nphi * a.nphi;
  const int lt = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  const int tri = a.tri0 + lt, nb = a.nb;
  const int b1 = tri / (nb * nb), b2 = (tri / nb) % nb, b3 = tri % nb;
  const double t1 = a.tb[b1], t2 = a.tb[b2], t3 = a.tb[b3];
  const double dphi = 2.0 * kPi / a.nphi;
  const double geo = 2.0 * kPi * t1 * t2 * t3 * a.vol[b1] * a.vol[b2] * a.vol[b3] * dphi * dphi;
  const size_t kbeg = nph2 * split / nsplit, kend = nph2 * (split + 1) / nsplit;
  for (int ia = threadIdx.x; ia < a.n_ap; ia += blockDim.x) {
    const double th2 = a.ap[ia] * a.ap[ia], h = 0.5 * th2;
    const double q0 = 4.0 * kPi * th2 * th2;
    const double norm = 1.0 / (q0 * q0 * q0 * q0);
    double f = 1.0, hh = h;
    for (int t = 0; t < 5; ++t) { if (t > 0) f *= t; hps[ia][t] = kPi * f * hh * norm; hh *= h; }
  }
  const int npairs = 8 * a.n_ap;
  double2 acc[kM4MaxPairs];
  for (int r = 0; r < kM4MaxPairs; ++r) acc[r] = make_double2(0, 0);
  for (size_t k0 = kbeg; k0 < kend; k0 += kM4Bins) {
    __syncthreads();  // previous tile fully consumed (and hps written)
    {
      // one (bin, mu) item per thread
      const int j = threadIdx.x >> 3, mu = threadIdx.x & 7;
      const size_t k = k0 + j;
      if (k >= kend) {
        for (int t = 0; t < 5; ++t) coef[j][mu][t] = make_double2(0, 0);
        if (mu == 0) sd2s[j] = 0;
      } else {
        const int p = (int)(k / a.nphi), q = (int)(k % a.nphi);
        const double p12 = (p + 0.5) * dphi, p13 = (q + 0.5) * dphi;
        double s12, c12, s13, c13;
        sincos(p12, &s12, &c12);
        sincos(p13, &s13, &c13);
        const double2 v[4] = {make_double2(0, 0), make_double2(t1, 0), make_double2(t2 * c12, t2 * s12),
                              make_double2(t3 * c13, t3 * s13)};
        const double2 cen =
            make_double2((v[1].x + v[2].x + v[3].x) * 0.25, (v[1].y + v[2].y + v[3].y) * 0.25);
        double2 d[4];
        double sd2 = 0;
        for (int jj = 0; jj < 4; ++jj) {
          d[jj] = make_double2(v[jj].x - cen.x, v[jj].y - cen.y);
          sd2 += d[jj].x * d[jj].x + d[jj].y * d[jj].y;
        }
        if (mu == 0) sd2s[j] = sd2;
        double2 P[9], R[9];
        int dP = 0, dR = 0;
        P[0] = make_double2(1, 0);
        R[0] = make_double2(1, 0);
        for (int jj = 0; jj < 4; ++jj) {
          const bool cj = kBeta[mu][jj];
          double2* poly = cj ? R : P;
          int& dg = cj ? dR : dP;
          const double2 root = cj ? d[jj] : make_double2(d[jj].x, -d[jj].y);
          for (int rep = 0; rep < 2; ++rep) {
            poly[dg + 1] = poly[dg];
            for (int t = dg; t >= 1; --t) {
              const double2 m = cm(poly[t], root);
              poly[t] = make_double2(poly[t - 1].x + m.x, poly[t - 1].y + m.y);
            }
            poly[0] = cm(poly[0], root);
            ++dg;
          }
        }
        // e^{i ph}, ph = 2 sum s_a zeta_a, zeta = (phi13/2, 0, phi12, phi13)
        const double ph = (kBeta[mu][0] ? -1.0 : 1.0) * p13 + 2.0 * (kBeta[mu][2] ? -1.0 : 1.0) * p12 +
                          2.0 * (kBeta[mu][3] ? -1.0 : 1.0) * p13;
        double sp, cp;
        sincos(ph, &sp, &cp);
        const double2 g =
            cm(gam[(size_t)mu * gam_mu_stride + (size_t)lt * nph2 + k], make_double2(cp * geo, sp * geo));
        const int tmax = dP < dR ? dP : dR;
        for (int t = 0; t < 5; ++t) coef[j][mu][t] = t <= tmax ? cm(g, cm(P[t], R[t])) : make_double2(0, 0);
      }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < kM4Bins * a.n_ap; w += blockDim.x) {
      const int j = w / a.n_ap, ia = w % a.n_ap;
      const double th = a.ap[ia];
      exs[j][ia] = exp(-sd2s[j] / (2.0 * th * th));
    }
    __syncthreads();
    for (int r = 0; r < kM4MaxPairs; ++r) {
      const int pr = threadIdx.x + r * kM4Threads;
      if (pr >= npairs) break;
      const int mu = pr / a.n_ap, ia = pr % a.n_ap;
      const int tmax = mu == 0 ? 0 : (mu < 5 ? 2 : 4);
      double2 s = acc[r];
      for (int j = 0; j < kM4Bins; ++j) {
        double re = 0, im = 0;
        for (int t = 0; t <= tmax; ++t) {
          re += coef[j][mu][t].x * hps[ia][t];
          im += coef[j][mu][t].y * hps[ia][t];
        }
        s.x += re * exs[j][ia];
        s.y += im * exs[j][ia];
      }
      acc[r] = s;
    }
  }
  for (int r = 0; r < kM4MaxPairs; ++r) {
    const int pr = threadIdx.x + r * kM4Threads;
    if (pr >= npairs) break;
    const int mu = pr / a.n_ap, ia = pr % a.n_ap;
    partial[(((size_t)tri * nsplit + split) * a.n_ap + ia) * 8 + mu] = acc[r];
  }
}

}  // namespace

cudaError_t real_space_counts(const double* ups, int nb, int N, int nphi, double* E_scratch,
                              int tri0, int ntri, double* norm_chunk, double* gam_chunk,
                              size_t gam_mu_stride, bool accumulate_into_existing, cudaStream_t s);

cudaError_t real_space(const double* ups, int nb, int N, int nphi, double* gamma, double* norm,
                       double* scratch_norm, double* E_scratch, cudaStream_t s) {
  const int nn = 2 * N + 1;
  const int ntri = nb * nb * nb;
  angle_table<<<64, 256, 0, s>>>(N, nphi, reinterpret_cast<double2*>(E_scratch));
  const size_t smem = (size_t)(nn * nn + nn * nphi) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(real_space_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(real_space_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const double2* U = reinterpret_cast<const double2*>(ups);
  const double2* E = reinterpret_cast<const double2*>(E_scratch);
  real_space_kernel<true><<<ntri, 256, smem, s>>>(U, nb, N, nphi, E, 0, ntri, nullptr, scratch_norm, nullptr, 0);
  const size_t stride = (size_t)ntri * nphi * nphi;
  real_space_kernel<false><<<8 * ntri, 256, smem, s>>>(U, nb, N, nphi, E, 0, ntri, scratch_norm, nullptr,
                                                       reinterpret_cast<double2*>(gamma), stride);
  add_arrays<<<1024, 256, 0, s>>>(norm, scratch_norm, stride);
  return cudaGetLastError();
}

size_t real_space_smem(int N, int nphi) {
  const int nn = 2 * N + 1;
  return (size_t)(nn * nn + nn * nphi) * sizeof(double2);
}

// Aperture measures: triples processed in chunks; returns per-(triple, slice, aperture)
// partial sums in `partial` [ntri][nsplit][n_ap][8] complex, the angular bins of each
// triple split into nsplit slices.
int map4_nsplit(int chunk_tri, int ntri, int n_ap) {
  int ns = (4 * 152 + chunk_tri - 1) / chunk_tri;
  const size_t cap = (size_t)(256u << 20) / ((size_t)ntri * n_ap * 8 * 16);
  if ((size_t)ns > cap) ns = (int)cap;
  return ns < 1 ? 1 : (ns > 16 ? 16 : ns);
}

cudaError_t map4_partials(const double* ups, const double* edges_host, int nb, int N, int nphi,
                          const double* ap_host, int n_ap, double* E_scratch, double* norm_chunk,
                          double* gam_chunk, int chunk_tri, int nsplit, double* partial, cudaStream_t s) {
  const int nn = 2 * N + 1;
  const int ntri = nb * nb * nb;
  angle_table<<<64, 256, 0, s>>>(N, nphi, reinterpret_cast<double2*>(E_scratch));
  ++g_launches;
  const size_t smem = (size_t)(nn * nn + nn * nphi) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(real_space_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(real_space_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Map4Args a;
  a.nb = nb; a.nphi = nphi; a.n_ap = n_ap;
  for (int b = 0; b < nb; ++b) {
    const double lo = edges_host[b], hi = edges_host[b + 1];
    a.tb[b] = (2.0 / 3.0) * (hi * hi * hi - lo * lo * lo) / (hi * hi - lo * lo);
    a.vol[b] = 0.5 * (hi * hi - lo * lo) / a.tb[b];
  }
  for (int k = 0; k < n_ap; ++k) a.ap[k] = ap_host[k];
  const double2* U = reinterpret_cast<const double2*>(ups);
  const double2* E = reinterpret_cast<const double2*>(E_scratch);
  const size_t nph2 = (size_t)nphi * nphi;
  for (int t0 = 0; t0 < ntri; t0 += chunk_tri) {
    const int nt = min(chunk_tri, ntri - t0);
    const size_t stride = (size_t)nt * nph2;
    cudaMemsetAsync(gam_chunk, 0, 8 * stride * sizeof(double2), s);
    real_space_kernel<true><<<nt, 256, smem, s>>>(U, nb, N, nphi, E, t0, nt, nullptr, norm_chunk, nullptr, 0);
    real_space_kernel<false><<<8 * nt, 256, smem, s>>>(U, nb, N, nphi, E, t0, nt, norm_chunk, nullptr,
                                                       reinterpret_cast<double2*>(gam_chunk), stride);
    a.tri0 = t0; a.ntri = nt;
    map4_kernel<<<nt * nsplit, kM4Threads, 0, s>>>(a, reinterpret_cast<const double2*>(gam_chunk), stride,
                                                   nsplit, reinterpret_cast<double2*>(partial));
    g_launches += 3;
  }
  return cudaGetLastError();
}

namespace {

// Sum the partials over triples and slices (fixed order), then the E/B split and the
// Gaussian part.
__global__ void map4_finish(const double2* __restrict__ partial, int nunits, int n_ap,
                            const double* __restrict__ xipm, const double* __restrict__ tb,
                            const double* __restrict__ area, int nb, const double* __restrict__ ap,
                            double* __restrict__ m4, double* __restrict__ eb, double* __restrict__ disc) {
  const int ia = blockIdx.x;
  __shared__ double2 mm[8];
  __shared__ double2 D[16];
  if (threadIdx.x < 8) {
    double re = 0, im = 0;
    for (int t = 0; t < nunits; ++t) {
      const double2 v = partial[((size_t)t * n_ap + ia) * 8 + threadIdx.x];
      re += v.x; im += v.y;
    }
    mm[threadIdx.x] = make_double2(re, im);
    m4[16 * ia + 2 * threadIdx.x] = re;
    m4[16 * ia + 2 * threadIdx.x + 1] = im;
  }
  __syncthreads();
  // all 16 conjugation patterns: the 8 computed ones and their complex conjugates
  if (threadIdx.x == 0) {
    for (int mu = 0; mu < 8; ++mu) {
      int code = 0, ccode = 0;
      for (int j = 0; j < 4; ++j) { code = 2 * code + kBeta[mu][j]; ccode = 2 * ccode + (1 - kBeta[mu][j]); }
      D[code] = mm[mu];
      D[ccode] = make_double2(mm[mu].x, -mm[mu].y);
    }
  }
  __syncthreads();
  // component c: bits of the label "t/x" for apertures 0..3 in the order of
  // Eq. 4PCF_rawcomponents (x = 1)
  const unsigned char lab[16] = {0x0, 0x8, 0x4, 0x2, 0x1, 0x3, 0x5, 0x6, 0x9, 0xA, 0xC, 0x7, 0xB, 0xD, 0xE, 0xF};
  if (threadIdx.x < 16) {
    const int c = threadIdx.x;
    double re = 0;
    for (int code = 0; code < 16; ++code) {
      // coefficient prod_a (t: 1/2; x: unconj -i/2, conj +i/2)
      double cr = 1, ci = 0;
      for (int j = 0; j < 4; ++j) {
        const bool isx = (lab[c] >> (3 - j)) & 1;
        const bool cj = (code >> (3 - j)) & 1;
        double fr, fi;
        if (!isx) { fr = 0.5; fi = 0; } else { fr = 0; fi = cj ? 0.5 : -0.5; }
        const double nr = cr * fr - ci * fi;
        ci = cr * fi + ci * fr;
        cr = nr;
      }
      re += cr * D[code].x - ci * D[code].y;
    }
    eb[16 * ia + c] = re;
  }
  __syncthreads();
  if (disc && xipm) {
    if (threadIdx.x == 0) {
      const double th = ap[ia];
      double Ar = 0, Ai = 0, Bp = 0;
      for (int b = 0; b < nb; ++b) {
        // xi_+ = sum x^* G_0 / sum w W_0, xi_- = sum x G_-4 / sum w W_0
        const double den = xipm[6 * b + 4];
        if (den == 0.0) continue;
        const double x = tb[b] / th, g = exp(-0.25 * x * x);
        const double Tp = (x * x * x * x - 16.0 * x * x + 32.0) / 128.0 * g;
        const double Tm = x * x * x * x / 128.0 * g;
        Bp += xipm[6 * b] / den * Tp * area[b] / (th * th);
        Ar += xipm[6 * b + 2] / den * Tm * area[b] / (th * th);
        Ai += xipm[6 * b + 3] / den * Tm * area[b] / (th * th);
      }
      for (int code = 0; code < 16; ++code) {
        int be[4];
        for (int j = 0; j < 4; ++j) be[j] = (code >> (3 - j)) & 1;
        double2 pr[4][4];
        for (int x = 0; x < 4; ++x)
          for (int y = 0; y < 4; ++y)
            pr[x][y] = (be[x] == be[y]) ? make_double2(Ar, be[x] ? -Ai : Ai) : make_double2(Bp, 0.0);
        const double2 a1 = cm(pr[0][1], pr[2][3]), a2 = cm(pr[0][2], pr[1][3]), a3 = cm(pr[0][3], pr[1][2]);
        D[code] = make_double2(a1.x + a2.x + a3.x, a1.y + a2.y + a3.y);
      }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      const int c = threadIdx.x;
      double re = 0;
      for (int code = 0; code < 16; ++code) {
        double cr = 1, ci = 0;
        for (int j = 0; j < 4; ++j) {
          const bool isx = (lab[c] >> (3 - j)) & 1;
          const bool cj = (code >> (3 - j)) & 1;
          double fr, fi;
          if (!isx) { fr = 0.5; fi = 0; } else { fr = 0; fi = cj ? 0.5 : -0.5; }
          const double nr = cr * fr - ci * fi;
          ci = cr * fi + ci * fr;
          cr = nr;
        }
        re += cr * D[code].x - ci * D[code].y;
      }
      disc[16 * ia + c] = re;
    }
  }
}

}  // namespace

cudaError_t map4_finish_launch(const double* partial, int ntri, int n_ap, const double* d_xipm,
                               const double* d_tb, const double* d_area, int nb, const double* d_ap,
                               double* d_m4, double* d_eb, double* d_disc, cudaStream_t s) {
  map4_finish<<<n_ap, 32, 0, s>>>(reinterpret_cast<const double2*>(partial), ntri, n_ap, d_xipm, d_tb,
                                  d_area, nb, d_ap, d_m4, d_eb, d_disc);
  ++g_launches;
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------
// Real-space transform that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being captured
// with a relaxed allocator policy, plug-ins whose host application owns all device memory,
// and real-time loops that must not block in the allocator.  For them this entry point
// keeps its scratch (the angular-bin table and the per-bin normalisation counts) in one
// file-scope device array of kStaticScratchBytes, held by every GPU that loads the library
// until the process exits.  Its address is looked up once per device with
// cudaGetSymbolAddress (the host symbol is only a stand-in and must not be passed to a
// kernel).  Every call shares the array: calls that overlap on the GPU race.  Both scratch
// regions are fully overwritten by each call before they are read, so nothing needs to be
// cleared.
// ---------------------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = 16u << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[64] = {};

// address of the static scratch on the current device (set-up on first use per device)
cudaError_t static_scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

bool device_resident(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

size_t real_space_smem(int N, int nphi);
cudaError_t real_space(const double* ups, int nb, int N, int nphi, double* gamma, double* norm,
                       double* scratch_norm, double* E_scratch, cudaStream_t s);

}  // namespace ext4pcf

extern "C" EXT4PCF_API int ext4pcf_to_real_space_noalloc(const double* upsilon, int n_bins, int n_max,
                                                         int n_phi, double* gamma, double* norm,
                                                         void* stream) {
  using namespace ext4pcf;
  if (!upsilon || !gamma || !norm) return EXT4PCF_E_INVALID_ARG;
  if (n_bins < 1 || n_bins > 32 || n_max < 0 || n_max > 40 || n_phi < 1 || n_phi > 1024)
    return EXT4PCF_E_INVALID_ARG;
  const size_t table_bytes = (size_t)(2 * n_max + 1) * n_phi * 16;
  const size_t norm_bytes = (size_t)n_bins * n_bins * n_bins * n_phi * n_phi * 8;
  const size_t table_off = (norm_bytes + 255) / 256 * 256;
  if (table_off + table_bytes > kStaticScratchBytes) return EXT4PCF_E_UNSUPPORTED;
  if (real_space_smem(n_max, n_phi) > 227 * 1024) return EXT4PCF_E_UNSUPPORTED;
  if (!device_resident(upsilon) || !device_resident(gamma) || !device_resident(norm))
    return EXT4PCF_E_INVALID_ARG;
  void* base = nullptr;
  if (static_scratch_ptr(&base) != cudaSuccess) return EXT4PCF_E_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaError_t e = real_space(upsilon, n_bins, n_max, n_phi, gamma, norm, reinterpret_cast<double*>(b),
                             reinterpret_cast<double*>(b + table_off), static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? EXT4PCF_OK : EXT4PCF_E_CUDA;
}
