// Factor table of the Khatri-Rao form of the 4PCF multipoles (Eq. 4PCFMultipoles with the
// natural components of Sec. 3.1), shared by the tensor-core contraction kernels.
//
// For fixed s = n2 + n3 every natural component factorises as
//   Upsilon_mu[n2,n3](Th1,Th2,Th3) = sum_i A_i^mu[s](Th1) * xt_i B_i[n2](Th2) C_i[n3](Th3).
// A row type fixes the centre factor xt, the row factors B, C and the one or two components
// (with their column factor A) that share the product xt B C.
#pragma once

namespace ext4pcf {
namespace {

struct KF {
  signed char arr, sgn, off, conj;  // arr 0: G, 1: W; index n = sgn * var + off
};
struct KRType {
  signed char xconj;  // 0: x, 1: x^*, 2: w
  KF B, C;            // row factors B(Th2; n2), C(Th3; n3)
  signed char nmu;
  signed char mu[2];
  KF A[2];            // column factors A(Th1; s)
};

// Khatri-Rao row types and the components that use them
#define EXT4PCF_KR_TABLE                                                                                  \
  {                                                                                                     \
    {0, {0, -1, -2, 0}, {0, -1, -3, 0}, 2, {0, 2}, {{0, 1, -3, 0}, {0, -1, -1, 1}}},                    \
    {0, {0, 1, -2, 1}, {0, -1, -3, 0}, 1, {3, 0}, {{0, 1, -3, 0}, {0, 0, 0, 0}}},                       \
    {0, {0, -1, -2, 0}, {0, 1, -1, 1}, 1, {4, 0}, {{0, 1, -3, 0}, {0, 0, 0, 0}}},                       \
    {1, {0, -1, -2, 0}, {0, -1, -1, 0}, 2, {1, 5}, {{0, 1, -1, 0}, {0, -1, -3, 1}}},                    \
    {1, {0, 1, -2, 1}, {0, -1, -1, 0}, 1, {6, 0}, {{0, 1, -1, 0}, {0, 0, 0, 0}}},                       \
    {1, {0, -1, -2, 0}, {0, 1, -3, 1}, 1, {7, 0}, {{0, 1, -1, 0}, {0, 0, 0, 0}}},                       \
    {2, {1, -1, 0, 0}, {1, -1, 0, 0}, 1, {8, 0}, {{1, 1, 0, 0}, {0, 0, 0, 0}}},                         \
  }
__constant__ KRType kKR[7] = EXT4PCF_KR_TABLE;
// host copy of the same initializer (inspection through ext4pcf_contraction_tables)
const KRType kKRHost[7] = EXT4PCF_KR_TABLE;
constexpr int kKRTypes = 7;

bool same_kf(KF a, KF b) { return a.arr == b.arr && a.sgn == b.sgn && a.off == b.off && a.conj == b.conj; }

// Partner mu' and offset o of every component under the exchange of Theta2 and Theta3, from
// the factor table: the centre factor and the column factor A(s) (s = n2 + n3 is kept) must be
// the same, and the row factors must trade places, B'(n3 + o) = C(n3) and C'(n2 - o) = B(n2).
// Returns false if a component has no partner.
bool derive_swap_map(signed char mup[9], signed char off[9]) {
  for (int mu = 0; mu < 9; ++mu) {
    int t = -1, g = 0;
    for (int k = 0; k < kKRTypes && t < 0; ++k)
      for (int j = 0; j < kKRHost[k].nmu; ++j)
        if (kKRHost[k].mu[j] == mu) { t = k; g = j; }
    if (t < 0) return false;
    const KRType& a = kKRHost[t];
    bool found = false;
    for (int k = 0; k < kKRTypes && !found; ++k)
      for (int j = 0; j < kKRHost[k].nmu && !found; ++j) {
        const KRType& b = kKRHost[k];
        if (b.xconj != a.xconj || !same_kf(b.A[j], a.A[g])) continue;
        for (int o = -1; o <= 1 && !found; ++o) {
          KF bB = b.B, bC = b.C;  // B'(n3 + o) = C(n3): sgn' = sgn_C, off' + sgn' o = off_C
          if (bB.arr != a.C.arr || bB.conj != a.C.conj || bB.sgn != a.C.sgn || bB.off + bB.sgn * o != a.C.off) continue;
          if (bC.arr != a.B.arr || bC.conj != a.B.conj || bC.sgn != a.B.sgn || bC.off - bC.sgn * o != a.B.off) continue;
          mup[mu] = b.mu[j];
          off[mu] = (signed char)o;
          found = true;
        }
      }
    if (!found) return false;
  }
  return true;
}

// offset o shared by the components of row type t (the rows of a type serve all its components)
int type_offset(int t, const signed char off[9]) {
  const int o = off[kKRHost[t].mu[0]];
  for (int j = 1; j < kKRHost[t].nmu; ++j)
    if (off[kKRHost[t].mu[j]] != o) return 99;
  return o;
}

// bin pair p -> (b2, b3), b2 <= b3, pairs in row-major order of (b2, b3)
__device__ __forceinline__ void pair_of(int p, int nb, int& b2, int& b3) {
  int b = 0, first = 0;
  while (p >= first + (nb - b)) {
    first += nb - b;
    ++b;
  }
  b2 = b;
  b3 = b + (p - first);
}

// The x~B rows of the transposed wave array per row type:
// 0: x G[-n2-2]   1: x G[n2-2]^*   2: x^* G[-n2-2]   3: x^* G[n2-2]^*   4: w W[-n2] (|n2| <= N)
constexpr int kXBTypes = 5;
__constant__ signed char kXBOfType[7] = {0, 1, 0, 2, 3, 2, 4};

}  // namespace
}  // namespace ext4pcf
