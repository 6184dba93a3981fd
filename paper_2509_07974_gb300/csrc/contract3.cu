// Third-order multipoles (the shear 3PCF, N = 3 of paper App. F) from the per-centre records
// of the neighbour gather, with the factor tables generated for order 3
// (ext4pcf_nth_order_factors) rather than written by hand:
//   Upsilon_{mu,n}(Theta1, Theta2) = sign sum_i t_i [F1(Theta1) F2(Theta2) - delta_{Theta1 Theta2} D],
// F_l = G_m, conj(G_m) or W_m with m = a n + b, and D the product of the two factors' terms of
// one and the same neighbour (their sum over the bin is XX, XA or WW of the record), which
// removes the triplets whose two neighbours coincide.  Records in FP64 or FP32, products and
// sums in FP64.  One thread per (component, n, Theta1, Theta2, slice of the wave's centres),
// each slice's centres summed in order; the slices' partial sums are then added in slice order.
#include <algorithm>
#include <cstdlib>

#include "common.cuh"

extern "C" int ext4pcf_nth_order_factors(int order, int mu, int* table, int cap);

namespace ext4pcf {
namespace {

struct F3 {
  int arr, conj, a, b;  // arr 0: G, 1: W; index m = a n + b
};
struct D3 {
  int arr, idx, conj;  // arr 0: XX, 1: XA, 2: WW
};
struct C3 {
  int sign, centre;  // centre 0: x_i, 1: x_i^*, 2: w_i
  F3 f[2];
  D3 d;
};
struct Table3 {
  C3 c[5];  // mu = 0..3, 4: normalisation
};

__device__ __forceinline__ double2 cj(double2 v) { return make_double2(v.x, -v.y); }
__device__ __forceinline__ double2 d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 d2(double2 v) { return v; }

template <typename Cx>
__device__ __forceinline__ double2 factor(const Cx* __restrict__ r, const Layout& L, const F3& f, int n, int b) {
  const int m = f.a * n + f.b;
  double2 v;
  if (f.arr == 0) v = d2(r[L.G(m, b)]);
  else v = m >= 0 ? d2(r[L.W(m, b)]) : cj(d2(r[L.W(-m, b)]));  // W_{-m} = W_m^*
  return f.conj ? cj(v) : v;
}

template <typename Cx>
__device__ __forceinline__ double2 same_galaxy(const Cx* __restrict__ r, const Layout& L, const D3& d, int b) {
  double2 v;
  if (d.arr == 0) v = d2(r[L.XX(d.idx, b)]);
  else if (d.arr == 1) v = d.idx >= 0 ? d2(r[L.XA(d.idx, b)]) : cj(d2(r[L.XA(-d.idx, b)]));
  else v = d.idx >= 0 ? d2(r[L.WW(d.idx, b)]) : cj(d2(r[L.WW(-d.idx, b)]));
  return d.conj ? cj(v) : v;
}

// block = (component and n, slice of the centres); thread = (Theta1, Theta2)
template <typename Cx>
__global__ void contract3_kernel(const Layout L, const Table3 tab, const Cx* __restrict__ rec,
                                 const Cx* __restrict__ xw, int T, int S, double2* __restrict__ part) {
  const int nn = 2 * L.N + 1, nb = L.nb;
  const int comp = blockIdx.x / S, sl = blockIdx.x % S;
  const int mu = comp / nn, n = comp % nn - L.N;
  const C3 c = tab.c[mu];
  const int i0 = (int)((long long)T * sl / S), i1 = (int)((long long)T * (sl + 1) / S);
  for (int p = threadIdx.x; p < nb * nb; p += blockDim.x) {
    const int b1 = p / nb, b2 = p % nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = i0; i < i1; ++i) {
      const Cx* r = rec + (size_t)i * L.rec;
      const double2 x = d2(xw[2 * (size_t)i]);
      const double2 t = c.centre == 2 ? d2(xw[2 * (size_t)i + 1]) : (c.centre == 1 ? cj(x) : x);
      double2 v = cmul(factor(r, L, c.f[0], n, b1), factor(r, L, c.f[1], n, b2));
      if (b1 == b2) {
        const double2 d = same_galaxy(r, L, c.d, b1);
        v.x -= d.x;
        v.y -= d.y;
      }
      acc = cadd(acc, cmul(t, v));
    }
    part[((size_t)sl * 5 * nn + comp) * nb * nb + p] = acc;
  }
}

// thread = output entry: the slices' partial sums in slice order, with the component's sign
__global__ void contract3_sum(const Layout L, const Table3 tab, int S, const double2* __restrict__ part,
                              double* __restrict__ ups3) {
  const int nn = 2 * L.N + 1, nb2 = L.nb * L.nb;
  const size_t total = (size_t)5 * nn * nb2;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(o / ((size_t)nn * nb2));
    double re = 0.0, im = 0.0;
    for (int sl = 0; sl < S; ++sl) {
      const double2 v = part[(size_t)sl * total + o];
      re += v.x;
      im += v.y;
    }
    ups3[2 * o] += tab.c[mu].sign * re;
    ups3[2 * o + 1] += tab.c[mu].sign * im;
  }
}

// m = a n + b over |n| <= N stays inside [lo, hi]
bool in_range(const F3& f, int N, int lo, int hi) {
  const int m1 = f.a * N + f.b, m2 = -f.a * N + f.b;
  return std::min(m1, m2) >= lo && std::max(m1, m2) <= hi;
}

// Order-3 tables from the generator, with the same-neighbour term of each component; false
// if a needed index lies outside the gather's record (Layout) for this N.
bool build_table3(int N, Table3& t) {
  for (int k = 0; k < 5; ++k) {
    const int mu = k < 4 ? k : -1;
    int raw[10];
    if (ext4pcf_nth_order_factors(3, mu, raw, 10) != 10) return false;
    C3& c = t.c[k];
    c.sign = raw[0];
    c.centre = raw[1];
    for (int l = 0; l < 2; ++l) c.f[l] = F3{raw[2 + 4 * l], raw[3 + 4 * l], raw[4 + 4 * l], raw[5 + 4 * l]};
    const F3 &f0 = c.f[0], &f1 = c.f[1];
    if (f0.arr != f1.arr) return false;
    if (f0.arr == 1) {  // w_j e^{i m0 phi} w_j e^{i m1 phi}
      // the same-galaxy term below is W W at the summed index, valid only when neither W
      // factor is conjugated; a table with a conjugated W factor is refused
      if (f0.conj || f1.conj) return false;
      if (f0.a + f1.a != 0) return false;
      c.d = D3{2, f0.b + f1.b, 0};
      if (!in_range(f0, N, -2 * N, 2 * N) || !in_range(f1, N, -2 * N, 2 * N) || std::abs(c.d.idx) > 2 * N)
        return false;
      continue;
    }
    if (f0.conj == f1.conj) {  // x_j^2 e^{i (m0 + m1) phi}, conjugated if both factors are
      if (f0.a + f1.a != 0) return false;
      c.d = D3{0, f0.b + f1.b, f0.conj};
      if (c.d.idx < -2 * N - 6 || c.d.idx > 2 * N - 2) return false;
    } else {  // |x_j|^2 e^{i (m_plain - m_conj) phi}
      const F3& pl = f0.conj ? f1 : f0;
      const F3& cn = f0.conj ? f0 : f1;
      if (pl.a - cn.a != 0) return false;
      c.d = D3{1, pl.b - cn.b, 0};
      if (std::abs(c.d.idx) > 2 * N + 2) return false;
    }
    if (!in_range(f0, N, -2 * N - 3, 2 * N - 1) || !in_range(f1, N, -2 * N - 3, 2 * N - 1)) return false;
  }
  return true;
}

}  // namespace

bool contract3_supported(int N) {
  Table3 t;
  return build_table3(N, t);
}

int contract3_slices(int T) { return std::max(1, std::min(32, T / 128)); }
size_t contract3_scratch_bytes(const Layout& L, int T) {
  return (size_t)contract3_slices(T) * 5 * (2 * L.N + 1) * L.nb * L.nb * sizeof(double2);
}

template <typename Cx>
cudaError_t contract3_wave(const Layout& L, const Cx* rec, const Cx* xw, int T, double* ups3, double2* scratch,
                           cudaStream_t s) {
  Table3 t;
  if (!build_table3(L.N, t)) return cudaErrorInvalidValue;
  if (T <= 0) return cudaSuccess;
  const int S = contract3_slices(T);
  contract3_kernel<Cx><<<5 * (2 * L.N + 1) * S, 128, 0, s>>>(L, t, rec, xw, T, S, scratch);
  contract3_sum<<<64, 256, 0, s>>>(L, t, S, scratch, ups3);
  g_launches += 2;
  return cudaGetLastError();
}
template cudaError_t contract3_wave<float2>(const Layout&, const float2*, const float2*, int, double*, double2*,
                                            cudaStream_t);
template cudaError_t contract3_wave<double2>(const Layout&, const double2*, const double2*, int, double*,
                                             double2*, cudaStream_t);

}  // namespace ext4pcf
