// Natural components of the shear N-point function and their multipole factorisation
// (paper App. F): the tables that a multipole estimator of order N contracts, generated
// from the sign matrix beta instead of written by hand.  Host code only (no GPU, no
// context); the 4PCF contraction kernels carry hand-written tables of the same form, which
// ext4pcf_contraction_tables exposes for comparison.
//
// Enumeration (App. F.1): p = 0, 1, ..., floor(N/2) conjugated shears; for each p the sets
// of conjugated positions in lexicographic order (the rightmost position advances first);
// for even N only the first half of the p = N/2 sets (the others are complex conjugates).
//
// Factorisation (App. F.2): in the x-projection the centre's shear is projected on
// zeta_0 = (phi_1 + phi_{N-1}) / 2 and the neighbour in bin l on zeta_l = phi_l; with the
// Fourier kernel exp(-i sum_{k>=2} n_k (phi_k - phi_1)) the phase of neighbour l is
// exp(i c_l phi_l), c_l an affine function of n.  A neighbour shear gamma_c gives G_{c_l}; a
// conjugated one gives conj(G_{-c_l}).  Each projection contributes a factor -1 (Eq.
// gammatx_def), (-1)^N in all.
#include <cstring>

#include "common.cuh"

namespace ext4pcf {
int contraction_table_cc(int* out);
int contraction_table_tc(int* out);
int contraction_swap_map(int* out);
}  // namespace ext4pcf

namespace {

constexpr int kMaxOrder = 16;

long long binomial(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Row mu of beta (+1 / -1 per position); false if mu is out of range.
bool beta_row(int order, int mu, int* beta) {
  int idx = 0;
  for (int p = 0; 2 * p <= order; ++p) {
    long long count = binomial(order, p);
    if (2 * p == order) count /= 2;
    if (mu >= idx + count) {
      idx += (int)count;
      continue;
    }
    // the (mu - idx)-th p-subset in lexicographic order
    int c[kMaxOrder];
    for (int i = 0; i < p; ++i) c[i] = i;
    for (int step = idx; step < mu; ++step) {
      int i = p - 1;
      while (i >= 0 && c[i] == order - p + i) --i;
      ++c[i];
      for (int j = i + 1; j < p; ++j) c[j] = c[j - 1] + 1;
    }
    for (int l = 0; l < order; ++l) beta[l] = 1;
    for (int i = 0; i < p; ++i) beta[c[i]] = -1;
    return true;
  }
  return false;
}

}  // namespace

extern "C" {

int ext4pcf_nth_order_components(int order, int* beta, int cap) {
  if (order < 2 || order > kMaxOrder) return EXT4PCF_E_INVALID_ARG;
  const int n = 1 << (order - 1);
  if (!beta) return n;
  if (cap < n * order) return EXT4PCF_E_INVALID_ARG;
  for (int mu = 0; mu < n; ++mu) beta_row(order, mu, beta + (size_t)mu * order);
  return n;
}

int ext4pcf_nth_order_factors(int order, int mu, int* table, int cap) {
  if (order < 2 || order > kMaxOrder) return EXT4PCF_E_INVALID_ARG;
  const int n_mu = 1 << (order - 1);
  if (mu < -1 || mu >= n_mu) return EXT4PCF_E_INVALID_ARG;
  const int row = order + 1;  // arr, conj, a_2 .. a_{N-1}, b
  const int size = 2 + (order - 1) * row;
  if (!table) return size;
  if (cap < size) return EXT4PCF_E_INVALID_ARG;
  const bool norm = mu < 0;
  int beta[kMaxOrder];
  if (!norm) beta_row(order, mu, beta);
  // phase of neighbour l (1..N-1): sum_k a[l][k] n_k + b[l], k = 2..N-1
  int a[kMaxOrder][kMaxOrder], b[kMaxOrder];
  std::memset(a, 0, sizeof(a));
  std::memset(b, 0, sizeof(b));
  for (int k = 2; k <= order - 1; ++k) {  // Fourier kernel exp(-i n_k (phi_k - phi_1))
    a[k][k] -= 1;
    a[1][k] += 1;
  }
  if (!norm) {
    b[1] -= beta[0];  // centre on zeta_0 = (phi_1 + phi_{N-1}) / 2
    b[order - 1] -= beta[0];
    for (int l = 1; l <= order - 1; ++l) b[l] -= 2 * beta[l];  // neighbour l on zeta_l = phi_l
  }
  table[0] = norm ? 1 : ((order & 1) ? -1 : 1);
  table[1] = norm ? 2 : (beta[0] < 0 ? 1 : 0);
  for (int l = 1; l <= order - 1; ++l) {
    int* t = table + 2 + (l - 1) * row;
    const bool cj = !norm && beta[l] < 0;  // conj(sum w gamma_c e^{-i c phi}) = conj(G_{-c})
    t[0] = norm ? 1 : 0;
    t[1] = cj ? 1 : 0;
    for (int k = 2; k <= order - 1; ++k) t[k] = cj ? -a[l][k] : a[l][k];
    t[order] = cj ? -b[l] : b[l];
  }
  return size;
}

int ext4pcf_contraction_tables(int which, int* table, int cap) {
  if (which < 0 || which > 2) return EXT4PCF_E_INVALID_ARG;
  const int size = which == 2 ? 18 : 9 * (2 + 3 * 5);
  if (!table) return size;
  if (cap < size) return EXT4PCF_E_INVALID_ARG;
  if (which == 2) return ext4pcf::contraction_swap_map(table);
  return which == 0 ? ext4pcf::contraction_table_cc(table) : ext4pcf::contraction_table_tc(table);
}

}  // extern "C"
