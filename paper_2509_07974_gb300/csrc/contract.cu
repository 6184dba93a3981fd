// Contraction of a wave of per-centre multipole records into the 4PCF multipoles
//   Upsilon_{mu,n}(Theta1,Theta2,Theta3) += sum_i xt_i A_i(Theta1) B_i(Theta2) C_i(Theta3)
// (paper Eq. 4PCFUpsilon0 and the seven equations after it; Eq. Nnmultipoles), and of the
// multiple-counting terms of Table tab:4PCFMCCorr (App. A.1).  CUDA-core version, templated
// on the arithmetic type: FP64 throughout, or FP32 within a wave with the wave totals added
// into the FP64 output.
#include "common.cuh"

namespace ext4pcf {

namespace {

// Which per-centre array a factor reads and how its index follows from (s, n2, n3).
enum Arr { kG = 0, kW = 1, kXX = 2, kXA = 3, kWW = 4 };
struct Factor {
  signed char arr, sgn, off, conj;
};
struct Comp {
  signed char xconj;  // 0: x_i, 1: x_i^*, 2: w_i
  Factor A, B, C;     // A(Theta1; s), B(Theta2; n2), C(Theta3; n3)
};

// Upsilon_0..7 (x-projection) and N: xt * A[s] * B[n2] * C[n3].
#define EXT4PCF_COMP_TABLE                                                          \
  {                                                                               \
    {0, {kG, 1, -3, 0}, {kG, -1, -2, 0}, {kG, -1, -3, 0}},                        \
    {1, {kG, 1, -1, 0}, {kG, -1, -2, 0}, {kG, -1, -1, 0}},                        \
    {0, {kG, -1, -1, 1}, {kG, -1, -2, 0}, {kG, -1, -3, 0}},                       \
    {0, {kG, 1, -3, 0}, {kG, 1, -2, 1}, {kG, -1, -3, 0}},                         \
    {0, {kG, 1, -3, 0}, {kG, -1, -2, 0}, {kG, 1, -1, 1}},                         \
    {1, {kG, -1, -3, 1}, {kG, -1, -2, 0}, {kG, -1, -1, 0}},                       \
    {1, {kG, 1, -1, 0}, {kG, 1, -2, 1}, {kG, -1, -1, 0}},                         \
    {1, {kG, 1, -1, 0}, {kG, -1, -2, 0}, {kG, 1, -3, 1}},                         \
    {2, {kW, 1, 0, 0}, {kW, -1, 0, 0}, {kW, -1, 0, 0}},                           \
  }
__constant__ Comp kComp[9] = EXT4PCF_COMP_TABLE;
// host copy of the same initializer (inspection through ext4pcf_contraction_tables)
const Comp kCompHost[9] = EXT4PCF_COMP_TABLE;

// Double-counting terms: xt * P(merged slots; bin Theta_a) * O(remaining slot; Theta_b).
// kind 0: Theta1 = Theta2 (index n3), kind 1: Theta1 = Theta3 (index n2),
// kind 2: Theta2 = Theta3 (index s).
struct Corr {
  Factor P, O;
};
__constant__ Corr kCorr[3][9] = {
    {// Theta1 = Theta2: P[n3], O = C(Theta3)[n3]
     {{kXX, 1, -5, 0}, {kG, -1, -3, 0}},
     {{kXX, 1, -3, 0}, {kG, -1, -1, 0}},
     {{kXA, 1, -1, 0}, {kG, -1, -3, 0}},
     {{kXA, 1, -1, 0}, {kG, -1, -3, 0}},
     {{kXX, 1, -5, 0}, {kG, 1, -1, 1}},
     {{kXA, 1, 1, 0}, {kG, -1, -1, 0}},
     {{kXA, 1, 1, 0}, {kG, -1, -1, 0}},
     {{kXX, 1, -3, 0}, {kG, 1, -3, 1}},
     {{kWW, 1, 0, 0}, {kW, -1, 0, 0}}},
    {// Theta1 = Theta3: P[n2], O = B(Theta2)[n2]
     {{kXX, 1, -6, 0}, {kG, -1, -2, 0}},
     {{kXX, 1, -2, 0}, {kG, -1, -2, 0}},
     {{kXA, 1, -2, 0}, {kG, -1, -2, 0}},
     {{kXX, 1, -6, 0}, {kG, 1, -2, 1}},
     {{kXA, 1, -2, 0}, {kG, -1, -2, 0}},
     {{kXA, 1, 2, 0}, {kG, -1, -2, 0}},
     {{kXX, 1, -2, 0}, {kG, 1, -2, 1}},
     {{kXA, 1, 2, 0}, {kG, -1, -2, 0}},
     {{kWW, 1, 0, 0}, {kW, -1, 0, 0}}},
    {// Theta2 = Theta3: P[s], O = A(Theta1)[s]
     {{kXX, -1, -5, 0}, {kG, 1, -3, 0}},
     {{kXX, -1, -3, 0}, {kG, 1, -1, 0}},
     {{kXX, -1, -5, 0}, {kG, -1, -1, 1}},
     {{kXA, -1, -1, 0}, {kG, 1, -3, 0}},
     {{kXA, -1, -1, 0}, {kG, 1, -3, 0}},
     {{kXX, -1, -3, 0}, {kG, -1, -3, 1}},
     {{kXA, -1, 1, 0}, {kG, 1, -1, 0}},
     {{kXA, -1, 1, 0}, {kG, 1, -1, 0}},
     {{kWW, -1, 0, 0}, {kW, 1, 0, 0}}}};
// Triple term: TR index per component (x^3 u^-8, x^3 u^-4, x^2x^* u^-4, x^2x^*, w^3)
__constant__ signed char kTriple[9] = {0, 1, 2, 2, 2, 3, 3, 3, 4};

template <typename Cx>
__device__ __forceinline__ Cx fetch(const Cx* __restrict__ rec, const Layout& L, Factor f, int var,
                                    int b) {
  const int n = f.sgn * var + f.off;
  Cx v;
  bool cj = f.conj != 0;
  switch (f.arr) {
    case kG: v = rec[L.G(n, b)]; break;
    case kXX: v = rec[L.XX(n, b)]; break;
    case kW: v = rec[L.W(n >= 0 ? n : -n, b)]; cj ^= (n < 0); break;
    case kXA: v = rec[L.XA(n >= 0 ? n : -n, b)]; cj ^= (n < 0); break;
    default: v = rec[L.WW(n >= 0 ? n : -n, b)]; cj ^= (n < 0); break;
  }
  return cj ? cconj(v) : v;
}

template <typename Cx>
__device__ __forceinline__ Cx centre_factor(const Cx* __restrict__ xw, int c, int xconj) {
  Cx x = xw[2 * (size_t)c];
  if (xconj == 1) return cconj(x);
  if (xconj == 2) return xw[2 * (size_t)c + 1];
  return x;
}

constexpr int kChunk = 32;
constexpr int kCorrChunk = 128;  // centres staged per pass of the correction kernel

// threads of a contraction block: one per (Theta2, Theta3), rounded up to whole warps
constexpr int contract_threads(int nbt) {
  return (nbt * nbt + 31) / 32 * 32 < 128 ? 128 : (nbt * nbt + 31) / 32 * 32;
}

// Block (mu, n2, n3); thread (b2, b3); registers hold Theta1 = 0..NBT-1.
template <typename R, int NBT>
__global__ void __launch_bounds__(contract_threads(NBT))
contract_cuda_core(const Layout L, const cplx_t<R>* __restrict__ rec, const cplx_t<R>* __restrict__ xw,
                   int T, const int* __restrict__ n_live, int w0, double* __restrict__ ups) {
  using Cx = cplx_t<R>;
  T = wave_centres(T, n_live, w0);
  if (T == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx* sx = reinterpret_cast<Cx*>(smem_raw);
  Cx* sA = sx + kChunk;
  Cx* sB = sA + kChunk * NBT;
  Cx* sC = sB + kChunk * NBT;
  const int N = L.N, nb = L.nb, nn = 2 * N + 1;
  const int mu = blockIdx.x / (nn * nn);
  const int n2 = (blockIdx.x / nn) % nn - N, n3 = blockIdx.x % nn - N, s = n2 + n3;
  const Comp cp = kComp[mu];
  const int tid = threadIdx.x;
  const int b2 = tid / nb, b3 = tid % nb;
  const bool active = tid < nb * nb;
  Cx acc[NBT];
#pragma unroll
  for (int k = 0; k < NBT; ++k) acc[k] = cmk<Cx>(R(0), R(0));
  for (int c0 = 0; c0 < T; c0 += kChunk) {
    const int nc = min(kChunk, T - c0);
    for (int k = tid; k < nc * (3 * nb + 1); k += blockDim.x) {
      const int cc = k / (3 * nb + 1), r = k % (3 * nb + 1);
      const Cx* rc = rec + (size_t)(c0 + cc) * L.rec;
      if (r == 0) sx[cc] = centre_factor(xw, c0 + cc, cp.xconj);
      else if (r <= nb) sA[cc * NBT + r - 1] = fetch(rc, L, cp.A, s, r - 1);
      else if (r <= 2 * nb) sB[cc * NBT + r - 1 - nb] = fetch(rc, L, cp.B, n2, r - 1 - nb);
      else sC[cc * NBT + r - 1 - 2 * nb] = fetch(rc, L, cp.C, n3, r - 1 - 2 * nb);
    }
    __syncthreads();
    if (active) {
      for (int cc = 0; cc < nc; ++cc) {
        const Cx kr = cmul(cmul(sx[cc], sB[cc * NBT + b2]), sC[cc * NBT + b3]);
#pragma unroll
        for (int k = 0; k < NBT; ++k) {
          if (k < nb) {
            const Cx a = sA[cc * NBT + k];
            acc[k].x += a.x * kr.x;  // separate multiply-adds: a sum of products would
            acc[k].x -= a.y * kr.y;  // cost an extra multiply and add
            acc[k].y += a.x * kr.y;
            acc[k].y += a.y * kr.x;
          }
        }
      }
    }
    __syncthreads();
  }
  if (active) {
    const size_t nb3 = (size_t)nb * nb * nb;
    const size_t base = (((size_t)mu * nn + (n2 + N)) * nn + (n3 + N)) * nb3 + (size_t)b2 * nb + b3;
#pragma unroll
    for (int k = 0; k < NBT; ++k) {
      if (k < nb) {
        double* o = ups + 2 * (base + (size_t)k * nb * nb);
        o[0] += (double)acc[k].x;
        o[1] += (double)acc[k].y;
      }
    }
  }
}

// Correction sums over the wave: block (mu, kind, index); thread (2x2 tile of (ba, bb), slice
// of the centres), or, for the triple term, threads over the centres.
template <typename R>
__device__ __forceinline__ void corrections_block(const Layout& L, const cplx_t<R>* __restrict__ rec,
                                                  const cplx_t<R>* __restrict__ xw, int T,
                                                  double* __restrict__ corr, unsigned char* smem_raw) {
  using Cx = cplx_t<R>;
  if (T == 0) return;
  const int N = L.N, nb = L.nb, nn = 2 * N + 1, ns = 4 * N + 1;
  const int per_mu = 2 * nn + ns;  // index rows of the three double-counting kinds
  const int mu = blockIdx.x / (per_mu + 1);
  const int row = blockIdx.x % (per_mu + 1);
  const int tid = threadIdx.x;
  const Comp cp = kComp[mu];
  const size_t nb2 = (size_t)nb * nb;
  const size_t mu_base = (size_t)mu * ((size_t)per_mu * nb2 + nb);
  if (row < per_mu) {
    int kind, var;
    if (row < nn) { kind = 0; var = row - N; }
    else if (row < 2 * nn) { kind = 1; var = row - nn - N; }
    else { kind = 2; var = row - 2 * nn - 2 * N; }
    const Corr cr = kCorr[kind][mu];
    // staged per centre: x~ P (bins padded to an even count with zeros) and O
    const int nt2 = (nb + 1) / 2, nbp = 2 * nt2;
    Cx* sP = reinterpret_cast<Cx*>(smem_raw);
    Cx* sO = sP + kCorrChunk * nbp;
    // thread = (2x2 tile of (ba, bb), slice of the chunk's centres)
    const int ntiles = nt2 * nt2;
    const int nslices = max(1, (int)blockDim.x / ntiles);
    const int tile = tid % ntiles, slice = tid / ntiles;
    const bool active = slice < nslices;
    const int ta = 2 * (tile / nt2), tb = 2 * (tile % nt2);
    // products in R; each chunk's partial sums (at most kCorrChunk / nslices centres) are
    // added into FP64 registers, so no R-precision sum runs over more than one chunk
    double acc64[2][2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) acc64[i][j][0] = acc64[i][j][1] = 0.0;
    for (int c0 = 0; c0 < T; c0 += kCorrChunk) {
      const int nc = min(kCorrChunk, T - c0);
      for (int k = tid; k < nc * 2 * nbp; k += blockDim.x) {
        const int cc = k / (2 * nbp), r = k % (2 * nbp);
        const Cx* rc = rec + (size_t)(c0 + cc) * L.rec;
        Cx v = cmk<Cx>(R(0), R(0));
        if (r < nbp) {
          if (r < nb) v = cmul(centre_factor(xw, c0 + cc, cp.xconj), fetch(rc, L, cr.P, var, r));
          sP[cc * nbp + r] = v;
        } else {
          if (r - nbp < nb) v = fetch(rc, L, cr.O, var, r - nbp);
          sO[cc * nbp + r - nbp] = v;
        }
      }
      __syncthreads();
      if (active) {
        Cx acc[2][2];
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) acc[i][j] = cmk<Cx>(R(0), R(0));
        for (int cc = slice; cc < nc; cc += nslices) {
          const Cx p0 = sP[cc * nbp + ta], p1 = sP[cc * nbp + ta + 1];
          const Cx o0 = sO[cc * nbp + tb], o1 = sO[cc * nbp + tb + 1];
          acc[0][0] = cadd(acc[0][0], cmul(p0, o0));
          acc[0][1] = cadd(acc[0][1], cmul(p0, o1));
          acc[1][0] = cadd(acc[1][0], cmul(p1, o0));
          acc[1][1] = cadd(acc[1][1], cmul(p1, o1));
        }
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) {
            acc64[i][j][0] += (double)acc[i][j].x;
            acc64[i][j][1] += (double)acc[i][j].y;
          }
      }
      __syncthreads();
    }
    // fixed-order sum over the slices (FP64)
    double2* red = reinterpret_cast<double2*>(smem_raw);  // [nslices][ntiles][4]
    if (active)
      for (int q = 0; q < 4; ++q)
        red[((size_t)slice * ntiles + tile) * 4 + q] = make_double2(acc64[q >> 1][q & 1][0], acc64[q >> 1][q & 1][1]);
    __syncthreads();
    for (int o = tid; o < nb * nb; o += blockDim.x) {
      const int ba = o / nb, bb = o % nb;
      const int t = (ba >> 1) * nt2 + (bb >> 1), q = (ba & 1) * 2 + (bb & 1);
      double re = 0, im = 0;
      for (int sl = 0; sl < nslices; ++sl) {
        const double2 v = red[((size_t)sl * ntiles + t) * 4 + q];
        re += v.x;
        im += v.y;
      }
      double* out = corr + 2 * (mu_base + (size_t)row * nb2 + o);
      out[0] += re;
      out[1] += im;
    }
  } else {
    // triple term: threads stride over the centres, each summing every bin, then a
    // fixed-order tree reduction over the threads (one bin at a time)
    const int k = kTriple[mu];
    double* red = reinterpret_cast<double*>(smem_raw);  // [2][blockDim]
    for (int b = 0; b < nb; ++b) {
      double ar = 0.0, ai = 0.0;  // products in R, summed in FP64
      for (int c = tid; c < T; c += blockDim.x) {
        const Cx v = cmul(centre_factor(xw, c, cp.xconj), rec[(size_t)c * L.rec + L.TR(k, b)]);
        ar += (double)v.x;
        ai += (double)v.y;
      }
      red[tid] = ar;
      red[blockDim.x + tid] = ai;
      __syncthreads();
      // fold the entries past the largest power of two first, then a tree (any block size)
      int p2 = 1;
      while (2 * p2 <= (int)blockDim.x) p2 *= 2;
      if (tid + p2 < (int)blockDim.x) {
        red[tid] += red[tid + p2];
        red[blockDim.x + tid] += red[blockDim.x + tid + p2];
      }
      __syncthreads();
      for (int st = p2 / 2; st > 0; st >>= 1) {
        if (tid < st) {
          red[tid] += red[tid + st];
          red[blockDim.x + tid] += red[blockDim.x + tid + st];
        }
        __syncthreads();
      }
      if (tid == 0) {
        double* o = corr + 2 * (mu_base + (size_t)per_mu * nb2 + b);
        o[0] += red[0];
        o[1] += red[blockDim.x];
      }
      __syncthreads();
    }
  }
}

// xi accumulators per bin: (sum conj(x) G_0, sum x G_-4, sum w W_0), FP64, fixed order.
template <typename R>
__device__ __forceinline__ void xi_block(const Layout& L, const cplx_t<R>* __restrict__ rec,
                                         const cplx_t<R>* __restrict__ xw, int T, double* __restrict__ xi,
                                         double (*red)[256]) {
  if (T == 0) return;
  const int b = blockIdx.x, tid = threadIdx.x;
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int c = tid; c < T; c += blockDim.x) {
    const cplx_t<R>* rc = rec + (size_t)c * L.rec;
    const double xr = xw[2 * (size_t)c].x, xim = xw[2 * (size_t)c].y, w = xw[2 * (size_t)c + 1].x;
    const double g0r = rc[L.G(0, b)].x, g0i = rc[L.G(0, b)].y;
    const double g4r = rc[L.G(-4, b)].x, g4i = rc[L.G(-4, b)].y;
    const double w0r = rc[L.W(0, b)].x, w0i = rc[L.W(0, b)].y;
    v[0] += xr * g0r + xim * g0i; v[1] += xr * g0i - xim * g0r;
    v[2] += xr * g4r - xim * g4i; v[3] += xr * g4i + xim * g4r;
    v[4] += w * w0r; v[5] += w * w0i;
  }
  for (int k = 0; k < 6; ++k) red[k][tid] = v[k];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st)
      for (int k = 0; k < 6; ++k) red[k][tid] += red[k][tid + st];
    __syncthreads();
  }
  if (tid < 6) xi[6 * b + tid] += red[tid][0];
  __syncthreads();
}

// Correction sums over a wave: block (mu, kind, index); each block takes the wave's segments
// in order and adds each one's sums into its slot (one writer per output: no atomics, fixed
// order)
template <typename R>
__global__ void __launch_bounds__(256, 8) corrections_kernel(const Layout L, const cplx_t<R>* __restrict__ rec,
                                                            const cplx_t<R>* __restrict__ xw, const WavePlan plan,
                                                            double* __restrict__ corr, size_t corr_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int si = 0; si < plan.nseg; ++si) {
    const WaveSeg& g = plan.seg[si];
    corrections_block<R>(L, rec + (size_t)g.off * L.rec, xw + 2 * (size_t)g.off, seg_live(g),
                         corr + (size_t)g.slot * corr_stride, smem_raw);
    __syncthreads();
  }
}

// xi accumulators of a wave: block = radial bin, segments in order into their slots
template <typename R>
__global__ void xi_kernel(const Layout L, const cplx_t<R>* __restrict__ rec, const cplx_t<R>* __restrict__ xw,
                          const WavePlan plan, double* __restrict__ xi) {
  __shared__ double red[6][256];
  for (int si = 0; si < plan.nseg; ++si) {
    const WaveSeg& g = plan.seg[si];
    xi_block<R>(L, rec + (size_t)g.off * L.rec, xw + 2 * (size_t)g.off, seg_live(g),
                xi + (size_t)g.slot * 6 * L.nb, red);
  }
}

__global__ void apply_corrections(const Layout L, const double* __restrict__ corr, double* __restrict__ ups) {
  const int N = L.N, nb = L.nb, nn = 2 * N + 1, ns = 4 * N + 1, per_mu = 2 * nn + ns;
  const size_t nb2 = (size_t)nb * nb, nb3 = nb2 * nb;
  const size_t total = (size_t)9 * nn * nn * nb3;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b3 = (int)(e % nb), b2 = (int)((e / nb) % nb), b1 = (int)((e / nb2) % nb);
    if (b1 != b2 && b1 != b3 && b2 != b3) continue;
    const size_t r = e / nb3;
    const int n3 = (int)(r % nn) - N, n2 = (int)((r / nn) % nn) - N, mu = (int)(r / ((size_t)nn * nn));
    const int s = n2 + n3;
    const double* cm = corr + 2 * ((size_t)mu * ((size_t)per_mu * nb2 + nb));
    double vr = 0, vi = 0;
    if (b1 == b2) { const double* t = cm + 2 * ((size_t)(n3 + N) * nb2 + (size_t)b1 * nb + b3); vr += t[0]; vi += t[1]; }
    if (b1 == b3) { const double* t = cm + 2 * ((size_t)(nn + n2 + N) * nb2 + (size_t)b1 * nb + b2); vr += t[0]; vi += t[1]; }
    if (b2 == b3) { const double* t = cm + 2 * ((size_t)(2 * nn + s + 2 * N) * nb2 + (size_t)b2 * nb + b1); vr += t[0]; vi += t[1]; }
    if (b1 == b2 && b1 == b3) { const double* t = cm + 2 * ((size_t)per_mu * nb2 + b1); vr -= 2.0 * t[0]; vi -= 2.0 * t[1]; }
    ups[2 * e] -= vr;
    ups[2 * e + 1] -= vi;
  }
}

template <typename R, int NBT>
cudaError_t launch_contract(const Layout& L, const cplx_t<R>* rec, const cplx_t<R>* xw, int T,
                            const int* n_live, int w0, double* ups, cudaStream_t s) {
  const int nn = 2 * L.N + 1;
  const int threads = contract_threads(NBT);
  const size_t smem = (size_t)kChunk * (1 + 3 * NBT) * sizeof(cplx_t<R>);
  cudaError_t e = cudaFuncSetAttribute(contract_cuda_core<R, NBT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contract_cuda_core<R, NBT><<<9 * nn * nn, threads, smem, s>>>(L, rec, xw, T, n_live, w0, ups);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t contract_wave(const Layout& L, const cplx_t<R>* rec, const cplx_t<R>* xw, int T,
                          const int* n_live, int w0, double* ups, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  if (L.nb <= 4) return launch_contract<R, 4>(L, rec, xw, T, n_live, w0, ups, s);
  if (L.nb <= 8) return launch_contract<R, 8>(L, rec, xw, T, n_live, w0, ups, s);
  if (L.nb <= 12) return launch_contract<R, 12>(L, rec, xw, T, n_live, w0, ups, s);
  if (L.nb <= 16) return launch_contract<R, 16>(L, rec, xw, T, n_live, w0, ups, s);
  if (L.nb <= 24) return launch_contract<R, 24>(L, rec, xw, T, n_live, w0, ups, s);
  if (L.nb <= 32) return launch_contract<R, 32>(L, rec, xw, T, n_live, w0, ups, s);
  return cudaErrorInvalidValue;
}

size_t corrections_size(const Layout& L) {
  const int nn = 2 * L.N + 1, ns = 4 * L.N + 1;
  return (size_t)2 * 9 * ((size_t)(2 * nn + ns) * L.nb * L.nb + L.nb);
}

template <typename R>
cudaError_t corrections_wave(const Layout& L, const cplx_t<R>* rec, const cplx_t<R>* xw, const WavePlan& plan,
                             double* corr, double* xi_acc, cudaStream_t s) {
  if (plan.total <= 0 || plan.nseg <= 0) return cudaSuccess;
  const int nn = 2 * L.N + 1, ns = 4 * L.N + 1;
  const int blocks = 9 * (2 * nn + ns + 1);
  // 192 threads (10 resident blocks per SM) let the 9 x (2(2N+1) + 4N+2) blocks of a wave
  // run in one round on 152 SMs; never fewer threads than 2x2 tiles of (b_a, b_b)
  const int ntiles = ((L.nb + 1) / 2) * ((L.nb + 1) / 2);
  const int threads = std::max(192, (ntiles + 31) / 32 * 32);
  const int nbp = 2 * ((L.nb + 1) / 2);
  const size_t smem = std::max(std::max((size_t)kCorrChunk * 2 * nbp * sizeof(cplx_t<R>),
                                        (size_t)threads * 4 * sizeof(double2)),
                               (size_t)2 * threads * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(corrections_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  corrections_kernel<R><<<blocks, threads, smem, s>>>(L, rec, xw, plan, corr, corrections_size(L));
  ++g_launches;
  if (xi_acc) {
    xi_kernel<R><<<L.nb, 256, 0, s>>>(L, rec, xw, plan, xi_acc);
    ++g_launches;
  }
  return cudaGetLastError();
}

cudaError_t corrections_apply(const Layout& L, const double* corr, double* ups, cudaStream_t s) {
  const int nn = 2 * L.N + 1;
  const size_t total = (size_t)9 * nn * nn * L.nb * L.nb * L.nb;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 65536) blocks = 65536;
  apply_corrections<<<blocks, 256, 0, s>>>(L, corr, ups);
  ++g_launches;
  return cudaGetLastError();
}

template cudaError_t contract_wave<float>(const Layout&, const float2*, const float2*, int, const int*, int, double*,
                                          cudaStream_t);
template cudaError_t contract_wave<double>(const Layout&, const double2*, const double2*, int, const int*, int, double*,
                                           cudaStream_t);
template cudaError_t corrections_wave<float>(const Layout&, const float2*, const float2*, const WavePlan&, double*,
                                             double*, cudaStream_t);
template cudaError_t corrections_wave<double>(const Layout&, const double2*, const double2*, const WavePlan&,
                                              double*, double*, cudaStream_t);

// kComp in the layout of ext4pcf_nth_order_factors at order 4: sign, centre code, then per
// bin (array, conj, coefficient of n2, coefficient of n3, constant); A reads s = n2 + n3.
int contraction_table_cc(int* out) {
  for (int mu = 0; mu < 9; ++mu) {
    const Comp& c = kCompHost[mu];
    int* t = out + mu * 17;
    t[0] = 1;
    t[1] = c.xconj;
    const Factor f[3] = {c.A, c.B, c.C};
    for (int l = 0; l < 3; ++l) {
      int* r = t + 2 + 5 * l;
      r[0] = f[l].arr == kW ? 1 : 0;
      r[1] = f[l].conj;
      r[2] = (l == 0 || l == 1) ? f[l].sgn : 0;
      r[3] = (l == 0 || l == 2) ? f[l].sgn : 0;
      r[4] = f[l].off;
    }
  }
  return 9 * 17;
}

}  // namespace ext4pcf

