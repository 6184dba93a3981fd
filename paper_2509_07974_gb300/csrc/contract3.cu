// Third-order multipoles (the shear 3PCF, N = 3 of paper App. F) from the per-centre records
// of the neighbour gather, with the factor tables generated for order 3
// (ext4pcf_nth_order_factors) rather than written by hand:
//   Upsilon_{mu,n}(Theta1, Theta2) = sign sum_i t_i [F1(Theta1) F2(Theta2) - delta_{Theta1 Theta2} D],
// F_l = G_m, conj(G_m) or W_m with m = a n + b, and D the product of the two factors' terms of
// one and the same neighbour (their sum over the bin is XX, XA or WW of the record), which
// removes the triplets whose two neighbours coincide.  FP64; one thread per
// (component, n, Theta1, Theta2), the wave's centres summed in order.
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

__device__ __forceinline__ double2 factor(const double2* __restrict__ r, const Layout& L, const F3& f, int n,
                                          int b) {
  const int m = f.a * n + f.b;
  double2 v;
  if (f.arr == 0) v = r[L.G(m, b)];
  else v = m >= 0 ? r[L.W(m, b)] : cj(r[L.W(-m, b)]);  // W_{-m} = W_m^*
  return f.conj ? cj(v) : v;
}

__device__ __forceinline__ double2 same_galaxy(const double2* __restrict__ r, const Layout& L, const D3& d,
                                               int b) {
  double2 v;
  if (d.arr == 0) v = r[L.XX(d.idx, b)];
  else if (d.arr == 1) v = d.idx >= 0 ? r[L.XA(d.idx, b)] : cj(r[L.XA(-d.idx, b)]);
  else v = d.idx >= 0 ? r[L.WW(d.idx, b)] : cj(r[L.WW(-d.idx, b)]);
  return d.conj ? cj(v) : v;
}

__global__ void contract3_kernel(const Layout L, const Table3 tab, const double2* __restrict__ rec,
                                 const double2* __restrict__ xw, int T, double* __restrict__ ups3) {
  const int nn = 2 * L.N + 1, nb = L.nb;
  const int mu = blockIdx.x / nn, n = blockIdx.x % nn - L.N;
  const C3 c = tab.c[mu];
  for (int p = threadIdx.x; p < nb * nb; p += blockDim.x) {
    const int b1 = p / nb, b2 = p % nb;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < T; ++i) {
      const double2* r = rec + (size_t)i * L.rec;
      const double2 x = xw[2 * (size_t)i];
      const double2 t = c.centre == 2 ? xw[2 * (size_t)i + 1] : (c.centre == 1 ? cj(x) : x);
      double2 v = cmul(factor(r, L, c.f[0], n, b1), factor(r, L, c.f[1], n, b2));
      if (b1 == b2) {
        const double2 d = same_galaxy(r, L, c.d, b1);
        v.x -= d.x;
        v.y -= d.y;
      }
      acc = cadd(acc, cmul(t, v));
    }
    double* o = ups3 + 2 * (((size_t)mu * nn + (n + L.N)) * nb * nb + p);
    o[0] += c.sign * acc.x;
    o[1] += c.sign * acc.y;
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

cudaError_t contract3_wave(const Layout& L, const double2* rec, const double2* xw, int T, double* ups3,
                           cudaStream_t s) {
  Table3 t;
  if (!build_table3(L.N, t)) return cudaErrorInvalidValue;
  if (T <= 0) return cudaSuccess;
  contract3_kernel<<<5 * (2 * L.N + 1), 128, 0, s>>>(L, t, rec, xw, T, ups3);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ext4pcf
