// Internal declarations shared by the CUDA translation units of libext4pcf.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "ext4pcf.h"

namespace ext4pcf {

// ---------------------------------------------------------------------------------------
// Complex helpers on float2 / double2 (re, im).
// ---------------------------------------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };
template <typename R> using cplx_t = typename C2<R>::T;

template <typename V> __host__ __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) {
  V v; v.x = a; v.y = b; return v;
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }

// ---------------------------------------------------------------------------------------
// Sizes of the per-centre multipole record (one centre, all radial bins).  Index ranges:
//   G  : n in [-2N-3, 2N-1]   sum_j x_j u^n            (x = w gamma_c, u = e^{i phi_ij})
//   W  : m in [0, 2N]         sum_j w_j u^m            (W_{-m} = conj W_m)
//   XX : n in [-2N-6, 2N-2]   sum_j x_j^2 u^n
//   XA : m in [0, 2N+2]       sum_j |x_j|^2 u^m        (conjugate-symmetric)
//   WW : m in [0, 2N]         sum_j w_j^2 u^m          (conjugate-symmetric)
//   TR : 5 values             x^3 u^-8, x^3 u^-4, x^2 x^* u^-4, x^2 x^*, w^3
// Each array is [n][nb] (bin fastest); the record is G|W|XX|XA|WW|TR.
// ---------------------------------------------------------------------------------------
struct Layout {
  int N, nb;
  int nG, nW, nXX, nXA;
  int oG, oW, oXX, oXA, oWW, oTR;  // complex-element offsets within a record
  int rec;                         // complex elements per centre record
  int max_pow;                     // largest |power| of u needed
  __host__ __device__ static Layout make(int N, int nb) {
    Layout L;
    L.N = N; L.nb = nb;
    L.nG = 4 * N + 3; L.nW = 2 * N + 1; L.nXX = 4 * N + 5; L.nXA = 2 * N + 3;
    L.oG = 0;
    L.oW = L.oG + L.nG * nb;
    L.oXX = L.oW + L.nW * nb;
    L.oXA = L.oXX + L.nXX * nb;
    L.oWW = L.oXA + L.nXA * nb;
    L.oTR = L.oWW + L.nW * nb;
    L.rec = L.oTR + 5 * nb;
    L.max_pow = 2 * N + 6;
    return L;
  }
  // element index of G_n(b), W_m(b) ... inside a record
  __host__ __device__ int G(int n, int b) const { return oG + (n + 2 * N + 3) * nb + b; }
  __host__ __device__ int W(int m, int b) const { return oW + m * nb + b; }
  __host__ __device__ int XX(int n, int b) const { return oXX + (n + 2 * N + 6) * nb + b; }
  __host__ __device__ int XA(int m, int b) const { return oXA + m * nb + b; }
  __host__ __device__ int WW(int m, int b) const { return oWW + m * nb + b; }
  __host__ __device__ int TR(int k, int b) const { return oTR + k * nb + b; }
};

// ---------------------------------------------------------------------------------------
// Cell grid of a catalogue.  The measure path computes it on the device (from the bounding
// box, without a host round trip) and the kernels read it from there; the direct aperture
// estimator chooses its own grid on the host.
// ---------------------------------------------------------------------------------------
struct GridGeom {
  double x0, y0;    // grid origin
  double cell;      // cell side (12 significant bits, so cx*cell is exact in float)
  double inv_cell;
  int ncx, ncy;     // cells per axis
  float cellf;
  int bad;          // 1 if the bounding box is not finite
};
// cells per axis never exceed this (the cell side is at least 1/4000 of the extent)
constexpr int kMaxCellsPerAxis = 4003;

// ---------------------------------------------------------------------------------------
// A catalogue sorted by cell (built by the grid kernels).
// ---------------------------------------------------------------------------------------
struct SortedCat {
  int n;            // galaxies
  const GridGeom* geom;  // device grid of the measure path (nullptr: the host fields below)
  int ncx, ncy;     // cells per axis
  double x0, y0;    // grid origin (double)
  double cell;      // cell side (few significant bits, so cx*cell is exact in float)
  float cellf;
  const int* cell_start;  // [ncx*ncy + 1]
  const int* perm;        // sorted position -> original index (within the catalogue)
  const double* px;       // sorted positions (double)
  const double* py;
  const double* xr;       // sorted x = w gamma_c (double), w
  const double* xi;
  const double* w;
  const float4* p4;       // (cx*cell, cy*cell, x - cx*cell, y - cy*cell) as float
  const float4* s4;       // (x_re, x_im, w, 0) as float
};

// kernels launched by this host thread (each launcher adds what it enqueues)
extern thread_local long long g_launches;

// Centres of a wave: at most T, and, when the catalogue's centre count is known only on the
// device (a centre mask), min(T, *n_live - w0) -- a wave past the end has none.
__device__ __forceinline__ int wave_centres(int T, const int* n_live, int w0) {
  if (!n_live) return T;
  const int left = *n_live - w0;
  return left < T ? (left > 0 ? left : 0) : T;
}

// A wave of the measure path: runs ("segments") of the centre lists of one or more catalogues,
// each at an offset of the wave's records that is a multiple of 64.  Centre lists and cell
// lists hold positions in the concatenated sorted arrays of all catalogues.
constexpr int kMaxSegs = 64;
struct WaveSeg {
  const int* centres;     // the catalogue's centre list
  const int* n_live;      // its length on the device (nullptr: t is exact)
  const GridGeom* geom;   // the catalogue's grid
  const int* cell_start;  // its cell list
  int w0;                 // first list index of the segment
  int t;                  // centres of the segment at most
  int off;                // first record of the segment in the wave
  int slot;               // output slot the segment accumulates into
  int cat;                // catalogue index
};
struct WavePlan {
  int nseg;
  int total;  // records of the wave: the last segment's off + t
  WaveSeg seg[kMaxSegs];
};
// live centres of a segment (device)
__device__ __forceinline__ int seg_live(const WaveSeg& g) { return wave_centres(g.t, g.n_live, g.w0); }
// segment holding record c, or -1 (records between segments are padding); *j = index in it
__device__ __forceinline__ int seg_of(const WavePlan& p, int c, int* j) {
  for (int s = p.nseg - 1; s >= 0; --s)
    if (c >= p.seg[s].off) {
      *j = c - p.seg[s].off;
      return *j < p.seg[s].t ? s : -1;
    }
  return -1;
}

struct Bins {
  int nb;
  double e2[65];   // squared edges (double)
  float e2f[65];   // squared edges (float)
  double rmax;
};

// ---------------------------------------------------------------------------------------
// Kernel launchers (implemented in the .cu files).
// ---------------------------------------------------------------------------------------
struct GridScratch;  // opaque, in grid.cu

// grid.cu: sort one catalogue (device arrays of n galaxies) into cells.  Writes the sorted
// arrays into caller-provided buffers and fills `out`.  Returns a cudaError_t.
struct GridBuffers {
  int* keys; int* keys_alt; int* perm; int* perm_alt; int* cell_start; size_t cell_cap;
  unsigned* hist; size_t hist_cap;
  double* px; double* py; double* xr; double* xi; double* w;
  float4* p4; float4* s4;
  double* bbox;  // [4] device
};
cudaError_t grid_bbox(const double* pos, int n, double* d_bbox, cudaStream_t s);
cudaError_t grid_sort(const double* pos, const double* shear, const double* wts, int n,
                      double x0, double y0, double cell, int ncx, int ncy, bool want_f32,
                      GridBuffers& gb, SortedCat& out, cudaStream_t s);
// the measure path: the grid chosen on the device from the bounding box d_bbox (written by
// grid_bbox) for separations up to rmax, then the sort.  The sorted arrays of gb point at this
// catalogue's place in the concatenated arrays, whose first galaxy is c0; the cell list holds
// concatenated positions and needs grid_cells_cap(n) entries; positions that are not finite
// set bit 1 of *status
cudaError_t grid_sort_device(const double* pos, const double* shear, const double* wts, int n, int c0,
                             const double* d_bbox, double rmax, GridGeom* d_geom, bool want_f32,
                             GridBuffers& gb, SortedCat& out, int* status, cudaStream_t s);
// Reduced catalogue of the tree approximation (Sect. 3.2, App. F.3): the galaxies of every
// non-empty cell of side delta, anchored at the lower corner of the bounding box d_bbox
// (grid_bbox), replaced by one galaxy at their weighted centre of mass carrying the summed w and
// w gamma.  Writes rpos [m][2], rshear [m][2] (summed w gamma / summed w, so that w * shear is
// the summed w gamma), rw [m] in cell order, and m to *count (device); head: n + 1 unsigned of
// scratch; a grid of more than kMaxCellsPerAxis cells per axis sets bit 4 of *status
cudaError_t reduce_catalogue(const double* pos, const double* shear, const double* wts, int n, const double* d_bbox,
                             double delta, GridGeom* d_geom, GridBuffers& gb, unsigned* head, double* rpos,
                             double* rshear, double* rw, int* count, int* status, cudaStream_t s);
// entries of a cell list of the measure path for n galaxies (the device grid keeps at most
// ~4n cells)
inline size_t grid_cells_cap(int64_t n) { return (size_t)(4 * n + 2); }

// Batched grid building: the catalogues of one measurement at once, concatenated.  c0[k] is
// the first galaxy of catalogue k (in the input and in the sorted arrays), coff[k] its first
// entry of the concatenated cell lists (grid_cells_cap entries each), tile0[k] / stile0[k] its
// first bounding-box / sort tile; c0[0] = coff[0] = tile0[0] = stile0[0] = 0.  The sort is
// segmented: every catalogue's keys are sorted in place within its range of positions.
constexpr int kMaxCatSet = 128;
constexpr int kBBoxTile = 8192;  // galaxies per bounding-box tile
constexpr int kSortTile = 2048;  // keys per radix-sort tile
struct CatSet {
  int n;
  int64_t c0[kMaxCatSet + 1];
  int64_t coff[kMaxCatSet + 1];
  int tile0[kMaxCatSet + 1];   // bounding-box tiles
  int stile0[kMaxCatSet + 1];  // radix-sort tiles (a tile never spans two catalogues)
};
// fills cs from the catalogue offsets (host); false if there are too many catalogues or cells
// for one set (then each catalogue is built on its own)
bool make_catset(const int64_t* c0, int n_cat, CatSet& cs);
// bounding boxes of every catalogue into bbox [n][4] (part: 4 doubles per tile of scratch)
cudaError_t bbox_batch(const double* pos, const CatSet& cs, double* part, double* bbox, cudaStream_t s);
// every catalogue's grid (the rule of grid_sort_device) and sorted arrays: gb's keys, perm and
// their alternates hold c0[n] entries, gb.cell_start the concatenated cell lists (coff), the
// sorted arrays c0[n] galaxies; perm (returned in *perm_out) maps a sorted position to its
// galaxy, both counted from the first galaxy of the set
cudaError_t grid_sort_batch(const double* pos, const double* shear, const double* wts, const CatSet& cs,
                            const double* bbox, double rmax, GridGeom* geoms, bool want_f32, GridBuffers& gb,
                            int** perm_out, int* status, cudaStream_t s);
// reduced catalogues (the rule of reduce_catalogue) of every catalogue, concatenated in
// catalogue order: catalogue k's m[k] reduced galaxies start at sum_{j<k} m[j]; counts[k] = m[k]
// (device); head: c0[n] + 1 unsigned of scratch
cudaError_t reduce_batch(const double* pos, const double* shear, const double* wts, const CatSet& cs,
                         const double* bbox, double delta, GridGeom* geoms, GridBuffers& gb, unsigned* head,
                         double* rpos, double* rshear, double* rw, int* counts, int* status, cudaStream_t s);

// gather.cu: per-centre multipole records of a wave (records of padding centres are left
// untouched).  cat: the neighbours' concatenated sorted arrays, whose grids the plan's segments
// give; cen: the arrays the centre lists index (the same, or the galaxies when the neighbours
// are a reduced catalogue); bins: the pass's bins (bins outside its range have zero width);
// accumulate: add into the records instead of writing them (and the centres' x, w)
template <typename R>
cudaError_t gather_wave(const SortedCat& cat, const SortedCat& cen, const Bins& bins, const Layout& L,
                        const WavePlan& plan, bool accumulate, cplx_t<R>* rec, cplx_t<R>* xw,
                        unsigned long long* pair_count, int sm_count, cudaStream_t s);

// contract.cu
template <typename R>
cudaError_t contract_wave(const Layout& L, const cplx_t<R>* rec, const cplx_t<R>* xw, int T,
                          const int* n_live, int w0, double* ups, cudaStream_t s);
// correction sums of every segment into its slot: corr + slot * corrections_size(L), and
// (xi_acc non-null) xi_acc + slot * 6 nb
template <typename R>
cudaError_t corrections_wave(const Layout& L, const cplx_t<R>* rec, const cplx_t<R>* xw, const WavePlan& plan,
                             double* corr, double* xi_acc, cudaStream_t s);
cudaError_t corrections_apply(const Layout& L, const double* corr, double* ups, cudaStream_t s);
size_t corrections_size(const Layout& L);  // doubles

// contract_tc.cu (tensor cores).  The wave is contracted into the reduced array of the
// Theta2 <-> Theta3 symmetry (tc_reduced_doubles doubles, zeroed per catalogue); tc_expand adds
// every ordered triple at |n| <= N from it into the output.  wave: the transposed wave array
// (contract_tc_xb_bytes); rowmax: the split-FP16 form's row maxima (contract_h16_rowmax_bytes).
bool tc_supported(const Layout& L, int precision);
cudaError_t contract_wave_tc(const Layout& L, const float2* rec, const float2* xw, int T,
                             const int* n_live, int w0, double* red, int precision, const int4* items,
                             int n_items, float2* wave, unsigned* rowmax, int* status, long long timeout,
                             cudaStream_t s);
size_t contract_tc_xb_bytes(const Layout& L, int T, int precision);
size_t tc_reduced_doubles(const Layout& L);
bool tc_build_items(const Layout& L, std::vector<int4>& items);
cudaError_t tc_expand(const Layout& L, const double* red, double* ups, cudaStream_t s);

// contract_h16.cu: the split-FP16 form
bool h16_supported(const Layout& L);
size_t contract_h16_wave_bytes(const Layout& L, int T);
size_t contract_h16_rowmax_bytes(const Layout& L);
// (plan: every segment's sums go to red + slot * tc_reduced_doubles(L))
cudaError_t contract_wave_h16(const Layout& L, const float2* rec, const float2* xw, const WavePlan& plan,
                              double* red, const int4* items, int n_items, float2* wave, unsigned* rowmax,
                              int* status, long long timeout, cudaStream_t s);

}  // namespace ext4pcf
