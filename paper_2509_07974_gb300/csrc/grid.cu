// Cell-list grid: every galaxy gets the key cy*ncx + cx of its cell, the (key, index) pairs
// are sorted with a stable least-significant-digit radix sort (8-bit digits), and the
// catalogue is rewritten in cell order.  The neighbour search of the gather kernel then
// reads each row of candidate cells as one contiguous range.
#include <cfloat>

#include "common.cuh"

namespace ext4pcf {

namespace {

constexpr int kTileThreads = 256;
constexpr int kTileItems = 8;  // keys per thread
constexpr int kTile = kTileThreads * kTileItems;

// ------------------------------------------------------------------------ bounding box
__global__ void bbox_partial(const double* __restrict__ pos, int n, double* __restrict__ part) {
  __shared__ double s[4][256];
  double mnx = DBL_MAX, mny = DBL_MAX, mxx = -DBL_MAX, mxy = -DBL_MAX;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x = pos[2 * i], y = pos[2 * i + 1];
    mnx = fmin(mnx, x); mxx = fmax(mxx, x);
    mny = fmin(mny, y); mxy = fmax(mxy, y);
  }
  s[0][threadIdx.x] = mnx; s[1][threadIdx.x] = mny; s[2][threadIdx.x] = mxx; s[3][threadIdx.x] = mxy;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + st]);
      s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + st]);
      s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + st]);
      s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void bbox_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double v[4] = {DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int b = 0; b < np; ++b) {
    v[0] = fmin(v[0], part[4 * b + 0]);
    v[1] = fmin(v[1], part[4 * b + 1]);
    v[2] = fmax(v[2], part[4 * b + 2]);
    v[3] = fmax(v[3], part[4 * b + 3]);
  }
  for (int k = 0; k < 4; ++k) out[k] = v[k];
}

// ------------------------------------------------------------------------ device grid
// cell side: about a sixteenth of the largest separation (finer cells leave fewer candidates
// outside the largest separation; 34 rows of cells at most), at most ~4000 cells per axis and
// about sqrt(n) per axis (so that the cells number at most 4n: grid_cells_cap), and with 12
// significant bits so that (cell index) * cell is exact in float
__device__ GridGeom make_geom(const double* __restrict__ bb, double rmax, int n) {
  GridGeom r;
  const bool finite = isfinite(bb[0]) && isfinite(bb[1]) && isfinite(bb[2]) && isfinite(bb[3]);
  r.bad = finite ? 0 : 1;
  const double x0 = finite ? bb[0] : 0.0, y0 = finite ? bb[1] : 0.0;
  const double wx = finite ? bb[2] - bb[0] : 0.0, wy = finite ? bb[3] - bb[1] : 0.0;
  const double extent = fmax(wx, wy);
  double c = rmax / 16.0;
  if (extent / 4000.0 > c) c = extent / 4000.0;
  // 1.01: the rounding to 12 bits below lowers c by less than 2^-12, so floor(extent / c)
  // stays below sqrt(n) and (sqrt(n) + 1)^2 <= 4n cells
  const double cn = 1.01 * extent / sqrt((double)(n > 0 ? n : 1));
  if (cn > c) c = cn;
  int ex;
  double m = frexp(c, &ex);          // c = m 2^ex, m in [0.5, 1)
  m = floor(m * 4096.0) / 4096.0;    // 12 significant bits
  c = ldexp(m, ex);
  r.x0 = x0;
  r.y0 = y0;
  r.cell = c;
  r.inv_cell = 1.0 / c;
  r.cellf = (float)c;
  r.ncx = min((int)floor(wx / c) + 1, kMaxCellsPerAxis);
  r.ncy = min((int)floor(wy / c) + 1, kMaxCellsPerAxis);
  return r;
}

__global__ void grid_geom_kernel(const double* __restrict__ bb, double rmax, int n, GridGeom* __restrict__ g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *g = make_geom(bb, rmax, n);
}

// the cell of a position in grid G (clamped into the grid)
__device__ __forceinline__ int cell_key(const GridGeom& G, double x, double y) {
  int cx = (int)floor((x - G.x0) * G.inv_cell);
  int cy = (int)floor((y - G.y0) * G.inv_cell);
  cx = min(max(cx, 0), G.ncx - 1);
  cy = min(max(cy, 0), G.ncy - 1);
  return cy * G.ncx + cx;
}

// a position that is not finite (NaN, which the bounding box's fmin/fmax skip, or +-inf)
// sets bit 1 of *status; its key is clamped into the grid like any other
__global__ void make_keys_dev(const double* __restrict__ pos, int n, const GridGeom* __restrict__ g,
                              int* __restrict__ keys, int* __restrict__ idx, int* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GridGeom G = *g;
  const double x = pos[2 * i], y = pos[2 * i + 1];
  if (!isfinite(x) || !isfinite(y)) atomicOr(status, 2);
  keys[i] = cell_key(G, x, y);
  idx[i] = i;
}

// ------------------------------------------------------------------------ keys
__global__ void make_keys(const double* __restrict__ pos, int n, double x0, double y0,
                          double inv_cell, int ncx, int ncy, int* __restrict__ keys,
                          int* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = (int)floor((pos[2 * i] - x0) * inv_cell);
  int cy = (int)floor((pos[2 * i + 1] - y0) * inv_cell);
  cx = min(max(cx, 0), ncx - 1);
  cy = min(max(cy, 0), ncy - 1);
  keys[i] = cy * ncx + cx;
  idx[i] = i;
}

// ------------------------------------------------------------------------ radix sort
static_assert(kTile == kSortTile, "sort tile");

// Tiles of a radix pass: tile t covers keys [base, base + cnt) and its count of digit d sits at
// hist[h0 + d * hstride] of the digit-major counts whose exclusive scan gives every digit run's
// first position.  One array: h0 = t, hstride = the tile count.  A catalogue set (segmented
// sort): the counts of catalogue k, digit-major over its own tiles, start at 256 stile0[k], so
// that the scan's offsets are positions inside catalogue k's own range.
struct PlainTiles {
  int n, ntiles;
  __device__ void tile(int t, int& base, int& cnt, size_t& h0, int& hstride) const {
    base = t * kTile;
    cnt = min(kTile, n - base);
    h0 = (size_t)t;
    hstride = ntiles;
  }
};
// largest k < n with v[k] <= x (empty catalogues share their start with the next one, which the
// search passes over)
__device__ __forceinline__ int seg_find(const int64_t* v, int n, int64_t x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (x >= v[mid]) lo = mid; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int seg_find(const int* v, int n, int x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (x >= v[mid]) lo = mid; else hi = mid;
  }
  return lo;
}
struct CatTiles {
  CatSet cs;
  __device__ void tile(int t, int& base, int& cnt, size_t& h0, int& hstride) const {
    const int k = seg_find(cs.stile0, cs.n, t);
    base = (int)cs.c0[k] + (t - cs.stile0[k]) * kTile;
    cnt = min(kTile, (int)cs.c0[k + 1] - base);
    hstride = cs.stile0[k + 1] - cs.stile0[k];
    h0 = (size_t)256 * cs.stile0[k] + (t - cs.stile0[k]);
  }
};

template <class Tiles>
__global__ void radix_hist(const int* __restrict__ keys, const Tiles tl, int shift, unsigned* __restrict__ hist) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base, cnt, hs;
  size_t h0;
  tl.tile(blockIdx.x, base, cnt, h0, hs);
  for (int k = 0; k < kTileItems; ++k) {
    const int j = k * kTileThreads + threadIdx.x;
    if (j < cnt) atomicAdd(&h[((unsigned)keys[base + j] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[h0 + (size_t)threadIdx.x * hs] = h[threadIdx.x];
}

// Stable scatter: warp w of a tile owns items [w*256, w*256+256) of the tile, visited in
// order in rounds of 32, so ranks follow input order.  The tile is first sorted by digit in
// shared memory; each digit's run is then written to its place in one contiguous, coalesced
// stretch (offs: exclusive scan of the digit counts, digit-major over the tiles).
template <class Tiles>
__global__ void radix_scatter(const int* __restrict__ keys_in, const int* __restrict__ val_in, const Tiles tl,
                              int shift, const unsigned* __restrict__ offs, int* __restrict__ keys_out,
                              int* __restrict__ val_out) {
  __shared__ unsigned wcnt[kTileThreads / 32][256];
  __shared__ unsigned dstart[256];  // first position of each digit in the tile's sorted order
  __shared__ unsigned wsum[kTileThreads / 32];
  __shared__ int skey[kTile];
  __shared__ int sval[kTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = threadIdx.x; d < (kTileThreads / 32) * 256; d += kTileThreads)
    (&wcnt[0][0])[d] = 0;
  __syncthreads();
  int tbase, tn, hs;
  size_t h0;
  tl.tile(blockIdx.x, tbase, tn, h0, hs);
  const int n = tbase + tn;  // items of the tile: [tbase, n)
  const int wbase = tbase + warp * (32 * kTileItems);
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kTileItems; ++r) {
    int i = wbase + r * 32 + lane;
    bool valid = i < n;
    unsigned valid_mask = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
      unsigned d = ((unsigned)keys_in[i] >> shift) & 0xFFu;
      unsigned peers = __match_any_sync(valid_mask, d);
      if ((peers & lt) == 0) wcnt[warp][d] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  {  // thread d: exclusive prefix over the warps of digit d, and the digit's tile total
    const unsigned d = threadIdx.x;
    unsigned run = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      const unsigned t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
    // exclusive scan of the totals over the digits (one per thread)
    unsigned inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    dstart[d] = before + inc - run;
    for (int w = 0; w < kTileThreads / 32; ++w) wcnt[w][d] += dstart[d];
  }
  __syncthreads();
  for (int r = 0; r < kTileItems; ++r) {
    int i = wbase + r * 32 + lane;
    bool valid = i < n;
    unsigned valid_mask = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
      int key = keys_in[i];
      unsigned d = ((unsigned)key >> shift) & 0xFFu;
      unsigned peers = __match_any_sync(valid_mask, d);
      unsigned pos = wcnt[warp][d] + __popc(peers & lt);
      skey[pos] = key;
      sval[pos] = val_in[i];
      __syncwarp(valid_mask);
      if ((peers & lt) == 0) wcnt[warp][d] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int j = threadIdx.x; j < tn; j += kTileThreads) {
    const int key = skey[j];
    const unsigned d = ((unsigned)key >> shift) & 0xFFu;
    const unsigned pos = offs[h0 + (size_t)d * hs] + ((unsigned)j - dstart[d]);
    keys_out[pos] = key;
    val_out[pos] = sval[j];
  }
}

// exclusive scan of unsigned values: block scan + recursive scan of block totals
constexpr int kScanBlock = 1024;

__global__ void scan_block(unsigned* __restrict__ data, size_t n, unsigned* __restrict__ totals) {
  __shared__ unsigned s[kScanBlock];
  size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
  unsigned v = i < n ? data[i] : 0u;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    unsigned t = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) data[i] = s[threadIdx.x] - v;
  if (threadIdx.x == kScanBlock - 1) totals[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_add(unsigned* __restrict__ data, size_t n, const unsigned* __restrict__ totals) {
  size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) data[i] += totals[blockIdx.x];
}

}  // namespace

cudaError_t scan_exclusive(unsigned* data, size_t n, unsigned* tmp, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t nb = (n + kScanBlock - 1) / kScanBlock;
  scan_block<<<(unsigned)nb, kScanBlock, 0, s>>>(data, n, tmp);
  ++g_launches;
  if (nb > 1) {
    cudaError_t e = scan_exclusive(tmp, nb, tmp + nb, s);
    if (e != cudaSuccess) return e;
    scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(data, n, tmp);
    ++g_launches;
  }
  return cudaGetLastError();
}

namespace {

// ------------------------------------------------------------------------ cell offsets
__global__ void cell_bounds(const int* __restrict__ keys, int n, int ncells, int* __restrict__ start) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  int lo = (p == 0) ? -1 : keys[p - 1];
  int hi = (p == n) ? ncells : keys[p];
  for (int c = lo + 1; c <= hi; ++c) start[c] = p;
}

// start[c] = c0 + first sorted position of cell c (c0: the catalogue's first galaxy in the
// concatenated arrays)
__global__ void cell_bounds_dev(const int* __restrict__ keys, int n, int c0, const GridGeom* __restrict__ g,
                                int* __restrict__ start) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  const int ncells = g->ncx * g->ncy;
  int lo = (p == 0) ? -1 : keys[p - 1];
  int hi = (p == n) ? ncells : keys[p];
  for (int c = lo + 1; c <= hi; ++c) start[c] = c0 + p;
}

__global__ void fill_start_empty(int* start, int ncells) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c <= ncells) start[c] = 0;
}

// ------------------------------------------------------------------------ sorted arrays
__global__ void build_sorted(const double* __restrict__ pos, const double* __restrict__ shear,
                             const double* __restrict__ wts, const int* __restrict__ perm,
                             const int* __restrict__ keys, int n, const GridGeom* __restrict__ geom,
                             int ncx, double x0, double y0,
                             double cell, float cellf, bool want_f32, double* __restrict__ px,
                             double* __restrict__ py, double* __restrict__ xr,
                             double* __restrict__ xi, double* __restrict__ w,
                             float4* __restrict__ p4, float4* __restrict__ s4) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i = perm[p];
  double x = pos[2 * i], y = pos[2 * i + 1], ww = wts[i];
  double gr = ww * shear[2 * i], gi = ww * shear[2 * i + 1];
  px[p] = x; py[p] = y; xr[p] = gr; xi[p] = gi; w[p] = ww;
  if (want_f32) {
    if (geom) {
      ncx = geom->ncx; x0 = geom->x0; y0 = geom->y0; cell = geom->cell; cellf = geom->cellf;
    }
    int key = keys[p];
    int cx = key % ncx, cy = key / ncx;
    // cx*cell and cy*cell are exact in float (cell has few significant bits)
    float ax = (float)cx * cellf, ay = (float)cy * cellf;
    float lx = (float)((x - x0) - (double)cx * cell);
    float ly = (float)((y - y0) - (double)cy * cell);
    p4[p] = make_float4(ax, ay, lx, ly);
    s4[p] = make_float4((float)gr, (float)gi, (float)ww, 0.f);
  }
}

}  // namespace

cudaError_t grid_bbox(const double* pos, int n, double* d_bbox, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int nblk = (n + 255) / 256;
  if (nblk > 512) nblk = 512;
  // partials go after the 4 result slots
  bbox_partial<<<nblk, 256, 0, s>>>(pos, n, d_bbox + 4);
  bbox_final<<<1, 32, 0, s>>>(d_bbox + 4, nblk, d_bbox);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t grid_sort(const double* pos, const double* shear, const double* wts, int n,
                      double x0, double y0, double cell, int ncx, int ncy, bool want_f32,
                      GridBuffers& gb, SortedCat& out, cudaStream_t s) {
  const int ncells = ncx * ncy;
  out.n = n; out.geom = nullptr; out.ncx = ncx; out.ncy = ncy; out.x0 = x0; out.y0 = y0;
  out.cell = cell; out.cellf = (float)cell;
  out.cell_start = gb.cell_start;
  out.perm = gb.perm;
  out.px = gb.px; out.py = gb.py; out.xr = gb.xr; out.xi = gb.xi; out.w = gb.w;
  out.p4 = gb.p4; out.s4 = gb.s4;
  if (n == 0) {
    fill_start_empty<<<(ncells + 256) / 256, 256, 0, s>>>(gb.cell_start, ncells);
    ++g_launches;
    return cudaGetLastError();
  }
  make_keys<<<(n + 255) / 256, 256, 0, s>>>(pos, n, x0, y0, 1.0 / cell, ncx, ncy, gb.keys, gb.perm);
  ++g_launches;
  int bits = 1;
  while ((1 << bits) < ncells) ++bits;
  const int ntiles = (n + kTile - 1) / kTile;
  int* kin = gb.keys; int* kout = gb.keys_alt;
  int* vin = gb.perm; int* vout = gb.perm_alt;
  unsigned* hist = gb.hist;
  unsigned* tmp = gb.hist + (size_t)256 * ntiles;
  const PlainTiles tl{n, ntiles};
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist<<<ntiles, kTileThreads, 0, s>>>(kin, tl, shift, hist);
    cudaError_t e = scan_exclusive(hist, (size_t)256 * ntiles, tmp, s);
    if (e != cudaSuccess) return e;
    radix_scatter<<<ntiles, kTileThreads, 0, s>>>(kin, vin, tl, shift, hist, kout, vout);
    g_launches += 2;  // histogram + scatter
    int* t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  out.perm = vin;
  cell_bounds<<<(n + 1 + 255) / 256, 256, 0, s>>>(kin, n, ncells, gb.cell_start);
  build_sorted<<<(n + 255) / 256, 256, 0, s>>>(pos, shear, wts, vin, kin, n, nullptr, ncx, x0, y0, cell,
                                               (float)cell, want_f32, gb.px, gb.py, gb.xr, gb.xi,
                                               gb.w, gb.p4, gb.s4);
  g_launches += 2;
  return cudaGetLastError();
}

namespace {
// stable LSD radix sort of (gb.keys, gb.perm) by keys below kMaxCellsPerAxis^2 < 2^24 (three
// 8-bit digits); *keys_out, *perm_out: where the sorted pairs ended up (ping-pong buffers)
cudaError_t radix_sort_cells(GridBuffers& gb, int n, int** keys_out, int** perm_out, cudaStream_t s) {
  const int ntiles = (n + kTile - 1) / kTile;
  int* kin = gb.keys; int* kout = gb.keys_alt;
  int* vin = gb.perm; int* vout = gb.perm_alt;
  unsigned* hist = gb.hist;
  unsigned* tmp = gb.hist + (size_t)256 * ntiles;
  const PlainTiles tl{n, ntiles};
  for (int shift = 0; shift < 24; shift += 8) {
    radix_hist<<<ntiles, kTileThreads, 0, s>>>(kin, tl, shift, hist);
    cudaError_t e = scan_exclusive(hist, (size_t)256 * ntiles, tmp, s);
    if (e != cudaSuccess) return e;
    radix_scatter<<<ntiles, kTileThreads, 0, s>>>(kin, vin, tl, shift, hist, kout, vout);
    g_launches += 2;
    int* t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  *keys_out = kin;
  *perm_out = vin;
  return cudaGetLastError();
}

// the segmented form: every catalogue of cs sorted within its own range of positions by
// keys below 2^24 (three passes); gb.hist holds 2 x 256 x stile0[n] + 4096 counters
cudaError_t radix_sort_cats(GridBuffers& gb, const CatSet& cs, int** keys_out, int** perm_out, cudaStream_t s) {
  const int ntiles = cs.stile0[cs.n];
  int* kin = gb.keys; int* kout = gb.keys_alt;
  int* vin = gb.perm; int* vout = gb.perm_alt;
  unsigned* hist = gb.hist;
  unsigned* tmp = gb.hist + (size_t)256 * ntiles;
  const CatTiles tl{cs};
  for (int shift = 0; shift < 24 && ntiles > 0; shift += 8) {
    radix_hist<<<ntiles, kTileThreads, 0, s>>>(kin, tl, shift, hist);
    cudaError_t e = scan_exclusive(hist, (size_t)256 * ntiles, tmp, s);
    if (e != cudaSuccess) return e;
    radix_scatter<<<ntiles, kTileThreads, 0, s>>>(kin, vin, tl, shift, hist, kout, vout);
    g_launches += 2;
    int* t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
  }
  *keys_out = kin;
  *perm_out = vin;
  return cudaGetLastError();
}

// grid of side delta anchored at the bounding box's lower corner (the tree approximation's
// resolution); more than kMaxCellsPerAxis cells per axis sets bit 4 of *status
__device__ GridGeom make_coarse_geom(const double* __restrict__ bb, double delta, int* __restrict__ status) {
  GridGeom r;
  const bool finite = isfinite(bb[0]) && isfinite(bb[1]) && isfinite(bb[2]) && isfinite(bb[3]);
  r.bad = finite ? 0 : 1;
  r.x0 = finite ? bb[0] : 0.0;
  r.y0 = finite ? bb[1] : 0.0;
  const double wx = finite ? bb[2] - bb[0] : 0.0, wy = finite ? bb[3] - bb[1] : 0.0;
  r.cell = delta;
  r.inv_cell = 1.0 / delta;
  r.cellf = (float)delta;
  const double cx = floor(wx / delta) + 1, cy = floor(wy / delta) + 1;
  if (cx > kMaxCellsPerAxis || cy > kMaxCellsPerAxis) atomicOr(status, 4);
  r.ncx = (int)fmin(cx, (double)kMaxCellsPerAxis);
  r.ncy = (int)fmin(cy, (double)kMaxCellsPerAxis);
  return r;
}

__global__ void coarse_geom_kernel(const double* __restrict__ bb, double delta, GridGeom* __restrict__ g,
                                   int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *g = make_coarse_geom(bb, delta, status);
}

// 1 at the first position of every run of equal sorted keys
__global__ void run_heads(const int* __restrict__ keys, int n, unsigned* __restrict__ head) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) head[p] = (p == 0 || keys[p] != keys[p - 1]) ? 1u : 0u;
}

// one thread per run (cell): the members in sorted order (a fixed summation order), their
// summed w, w gamma and w theta; the reduced galaxy sits at the weighted centre of mass
__global__ void reduce_runs(const int* __restrict__ keys, const int* __restrict__ perm,
                            const unsigned* __restrict__ head_scan, int n, const double* __restrict__ pos,
                            const double* __restrict__ shear, const double* __restrict__ wts,
                            double* __restrict__ rpos, double* __restrict__ rshear, double* __restrict__ rw,
                            int* __restrict__ count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (p == n - 1) *count = (int)head_scan[p] + ((p == 0 || keys[p] != keys[p - 1]) ? 1 : 0);
  if (!(p == 0 || keys[p] != keys[p - 1])) return;
  const int key = keys[p];
  double W = 0.0, Xr = 0.0, Xi = 0.0, Sx = 0.0, Sy = 0.0;
  for (int q = p; q < n && keys[q] == key; ++q) {
    const int i = perm[q];
    const double w = wts[i];
    W += w;
    Xr += w * shear[2 * i];
    Xi += w * shear[2 * i + 1];
    Sx += w * pos[2 * i];
    Sy += w * pos[2 * i + 1];
  }
  const unsigned r = head_scan[p];
  if (W != 0.0) {
    rpos[2 * r] = Sx / W;
    rpos[2 * r + 1] = Sy / W;
    rshear[2 * r] = Xr / W;  // w * shear gives back the summed w gamma
    rshear[2 * r + 1] = Xi / W;
  } else {
    const int i = perm[p];
    rpos[2 * r] = pos[2 * i];
    rpos[2 * r + 1] = pos[2 * i + 1];
    rshear[2 * r] = 0.0;
    rshear[2 * r + 1] = 0.0;
  }
  rw[r] = W;
}
}  // namespace

cudaError_t reduce_catalogue(const double* pos, const double* shear, const double* wts, int n, const double* d_bbox,
                             double delta, GridGeom* d_geom, GridBuffers& gb, unsigned* head, double* rpos,
                             double* rshear, double* rw, int* count, int* status, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(count, 0, sizeof(int), s);
  coarse_geom_kernel<<<1, 32, 0, s>>>(d_bbox, delta, d_geom, status);
  make_keys_dev<<<(n + 255) / 256, 256, 0, s>>>(pos, n, d_geom, gb.keys, gb.perm, status);
  g_launches += 2;
  int* keys = nullptr;
  int* perm = nullptr;
  cudaError_t e = radix_sort_cells(gb, n, &keys, &perm, s);
  if (e != cudaSuccess) return e;
  run_heads<<<(n + 255) / 256, 256, 0, s>>>(keys, n, head);
  e = scan_exclusive(head, (size_t)n, gb.hist, s);
  if (e != cudaSuccess) return e;
  reduce_runs<<<(n + 255) / 256, 256, 0, s>>>(keys, perm, head, n, pos, shear, wts, rpos, rshear, rw, count);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t grid_sort_device(const double* pos, const double* shear, const double* wts, int n, int c0,
                             const double* d_bbox, double rmax, GridGeom* d_geom, bool want_f32,
                             GridBuffers& gb, SortedCat& out, int* status, cudaStream_t s) {
  out.n = n;
  out.geom = d_geom;
  out.ncx = out.ncy = 0;
  out.x0 = out.y0 = out.cell = 0.0;
  out.cellf = 0.f;
  out.cell_start = gb.cell_start;
  out.perm = gb.perm;
  out.px = gb.px; out.py = gb.py; out.xr = gb.xr; out.xi = gb.xi; out.w = gb.w;
  out.p4 = gb.p4; out.s4 = gb.s4;
  if (n == 0) return cudaSuccess;
  grid_geom_kernel<<<1, 32, 0, s>>>(d_bbox, rmax, n, d_geom);
  make_keys_dev<<<(n + 255) / 256, 256, 0, s>>>(pos, n, d_geom, gb.keys, gb.perm, status);
  g_launches += 2;
  int* kin = nullptr;
  int* vin = nullptr;
  cudaError_t e0 = radix_sort_cells(gb, n, &kin, &vin, s);
  if (e0 != cudaSuccess) return e0;
  out.perm = vin;
  cell_bounds_dev<<<(n + 1 + 255) / 256, 256, 0, s>>>(kin, n, c0, d_geom, gb.cell_start);
  build_sorted<<<(n + 255) / 256, 256, 0, s>>>(pos, shear, wts, vin, kin, n, d_geom, 0, 0.0, 0.0, 1.0, 1.f,
                                               want_f32, gb.px, gb.py, gb.xr, gb.xi, gb.w, gb.p4, gb.s4);
  g_launches += 2;
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ batched forms
namespace {

// one block per tile of kBBoxTile galaxies of one catalogue
__global__ void bbox_tiles(const double* __restrict__ pos, const CatSet cs, double* __restrict__ part) {
  __shared__ double sm[4][256];
  const int t = blockIdx.x, k = seg_find(cs.tile0, cs.n, t);
  const int64_t a = cs.c0[k] + (int64_t)(t - cs.tile0[k]) * kBBoxTile;
  const int64_t b = min(a + kBBoxTile, cs.c0[k + 1]);
  double mnx = DBL_MAX, mny = DBL_MAX, mxx = -DBL_MAX, mxy = -DBL_MAX;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    const double x = pos[2 * i], y = pos[2 * i + 1];
    mnx = fmin(mnx, x); mxx = fmax(mxx, x);
    mny = fmin(mny, y); mxy = fmax(mxy, y);
  }
  sm[0][threadIdx.x] = mnx; sm[1][threadIdx.x] = mny; sm[2][threadIdx.x] = mxx; sm[3][threadIdx.x] = mxy;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sm[0][threadIdx.x] = fmin(sm[0][threadIdx.x], sm[0][threadIdx.x + st]);
      sm[1][threadIdx.x] = fmin(sm[1][threadIdx.x], sm[1][threadIdx.x + st]);
      sm[2][threadIdx.x] = fmax(sm[2][threadIdx.x], sm[2][threadIdx.x + st]);
      sm[3][threadIdx.x] = fmax(sm[3][threadIdx.x], sm[3][threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 4) part[4 * (size_t)t + threadIdx.x] = sm[threadIdx.x][0];
}

// thread k: catalogue k's bounding box from its tiles
__global__ void bbox_cats(const CatSet cs, const double* __restrict__ part, double* __restrict__ bbox) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cs.n) return;
  double v[4] = {DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int t = cs.tile0[k]; t < cs.tile0[k + 1]; ++t) {
    v[0] = fmin(v[0], part[4 * (size_t)t + 0]);
    v[1] = fmin(v[1], part[4 * (size_t)t + 1]);
    v[2] = fmax(v[2], part[4 * (size_t)t + 2]);
    v[3] = fmax(v[3], part[4 * (size_t)t + 3]);
  }
  for (int q = 0; q < 4; ++q) bbox[4 * k + q] = v[q];
}

// thread k: catalogue k's grid, for separations up to rmax (rmax > 0) or of side delta (the
// tree approximation's reduced catalogues: rmax <= 0)
__global__ void geom_cats(const CatSet cs, const double* __restrict__ bbox, double rmax, double delta,
                          GridGeom* __restrict__ geoms, int* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cs.n) return;
  const int n = (int)(cs.c0[k + 1] - cs.c0[k]);
  if (n == 0) return;
  geoms[k] = rmax > 0.0 ? make_geom(bbox + 4 * k, rmax, n) : make_coarse_geom(bbox + 4 * k, delta, status);
}

// keys of the set: every galaxy's cell in its catalogue's grid (below 2^24: at most
// kMaxCellsPerAxis^2 cells), sorted within the catalogue's range of positions
__global__ void keys_cats(const double* __restrict__ pos, const CatSet cs, const GridGeom* __restrict__ geoms,
                          int* __restrict__ keys, int* __restrict__ idx, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cs.c0[cs.n]) return;
  const int k = seg_find(cs.c0, cs.n, i);
  const double x = pos[2 * i], y = pos[2 * i + 1];
  if (!isfinite(x) || !isfinite(y)) atomicOr(status, 2);
  keys[i] = cell_key(geoms[k], x, y);
  idx[i] = (int)i;
}

// cell lists of the set from the sorted keys: thread p fills the entries between the cells of
// sorted positions p - 1 and p with p (the first galaxy at or after them), within the used
// part of each catalogue's list (ncx * ncy cells and the end entry)
__global__ void cell_bounds_cats(const int* __restrict__ keys, const CatSet cs, const GridGeom* __restrict__ geoms,
                                 int* __restrict__ start) {
  const int64_t n = cs.c0[cs.n];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  const int kl = p == 0 ? -1 : seg_find(cs.c0, cs.n, p - 1);  // catalogues of positions p - 1, p
  const int kh = p == n ? cs.n : seg_find(cs.c0, cs.n, p);
  const int lo = p == 0 ? -1 : keys[p - 1];
  const int hi = p == n ? -1 : keys[p];
  if (kl == kh) {
    int* st = start + cs.coff[kl];
    for (int c = lo + 1; c <= hi; ++c) st[c] = (int)p;
    return;
  }
  if (kl >= 0) {  // the rest of catalogue kl's list, its end entry included
    int* st = start + cs.coff[kl];
    const int end = geoms[kl].ncx * geoms[kl].ncy;
    for (int c = lo + 1; c <= end; ++c) st[c] = (int)p;
  }
  if (kh < cs.n) {  // catalogue kh's list up to its first galaxy's cell
    int* st = start + cs.coff[kh];
    for (int c = 0; c <= hi; ++c) st[c] = (int)p;
  }
}

__global__ void build_sorted_cats(const double* __restrict__ pos, const double* __restrict__ shear,
                                  const double* __restrict__ wts, const int* __restrict__ perm,
                                  const int* __restrict__ keys, const CatSet cs, const GridGeom* __restrict__ geoms,
                                  bool want_f32, double* __restrict__ px, double* __restrict__ py,
                                  double* __restrict__ xr, double* __restrict__ xi, double* __restrict__ w,
                                  float4* __restrict__ p4, float4* __restrict__ s4) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cs.c0[cs.n]) return;
  const int i = perm[p];
  const double x = pos[2 * (size_t)i], y = pos[2 * (size_t)i + 1], ww = wts[i];
  const double gr = ww * shear[2 * (size_t)i], gi = ww * shear[2 * (size_t)i + 1];
  px[p] = x; py[p] = y; xr[p] = gr; xi[p] = gi; w[p] = ww;
  if (want_f32) {
    const int k = seg_find(cs.c0, cs.n, p);
    const GridGeom G = geoms[k];
    const int key = keys[p];
    const int cx = key % G.ncx, cy = key / G.ncx;
    // cx*cell and cy*cell are exact in float (cell has few significant bits)
    const float ax = (float)cx * G.cellf, ay = (float)cy * G.cellf;
    const float lx = (float)((x - G.x0) - (double)cx * G.cell);
    const float ly = (float)((y - G.y0) - (double)cy * G.cell);
    p4[p] = make_float4(ax, ay, lx, ly);
    s4[p] = make_float4((float)gr, (float)gi, (float)ww, 0.f);
  }
}

// 1 at the first position of every run of equal keys inside one catalogue
__global__ void run_heads_cats(const int* __restrict__ keys, const CatSet cs, unsigned* __restrict__ head) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cs.c0[cs.n]) return;
  head[p] = (p == 0 || keys[p] != keys[p - 1] || seg_find(cs.c0, cs.n, p) != seg_find(cs.c0, cs.n, p - 1)) ? 1u
                                                                                                          : 0u;
}

// one thread per run (a cell of one catalogue): the rule of reduce_runs within the catalogue
__global__ void reduce_runs_cats(const int* __restrict__ keys, const int* __restrict__ perm,
                                 const unsigned* __restrict__ head_scan, const CatSet cs,
                                 const double* __restrict__ pos, const double* __restrict__ shear,
                                 const double* __restrict__ wts, double* __restrict__ rpos,
                                 double* __restrict__ rshear, double* __restrict__ rw) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cs.c0[cs.n]) return;
  const int k = seg_find(cs.c0, cs.n, p);
  if (!(p == cs.c0[k] || keys[p] != keys[p - 1])) return;
  const int key = keys[p];
  const int64_t end = cs.c0[k + 1];
  double W = 0.0, Xr = 0.0, Xi = 0.0, Sx = 0.0, Sy = 0.0;
  for (int64_t q = p; q < end && keys[q] == key; ++q) {
    const int i = perm[q];
    const double w = wts[i];
    W += w;
    Xr += w * shear[2 * (size_t)i];
    Xi += w * shear[2 * (size_t)i + 1];
    Sx += w * pos[2 * (size_t)i];
    Sy += w * pos[2 * (size_t)i + 1];
  }
  const unsigned r = head_scan[p];
  if (W != 0.0) {
    rpos[2 * (size_t)r] = Sx / W;
    rpos[2 * (size_t)r + 1] = Sy / W;
    rshear[2 * (size_t)r] = Xr / W;  // w * shear gives back the summed w gamma
    rshear[2 * (size_t)r + 1] = Xi / W;
  } else {
    const int i = perm[p];
    rpos[2 * (size_t)r] = pos[2 * (size_t)i];
    rpos[2 * (size_t)r + 1] = pos[2 * (size_t)i + 1];
    rshear[2 * (size_t)r] = 0.0;
    rshear[2 * (size_t)r + 1] = 0.0;
  }
  rw[r] = W;
}

// thread k: catalogue k's reduced galaxies, the runs of equal keys that start in its range of
// sorted positions (head_scan: exclusive scan of the run heads)
__global__ void run_counts(const unsigned* __restrict__ head_scan, const int* __restrict__ keys, const CatSet cs,
                           int* __restrict__ counts) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cs.n) return;
  const int64_t n = cs.c0[cs.n], a = cs.c0[k], b = cs.c0[k + 1];
  if (a == b) {
    counts[k] = 0;
    return;
  }
  auto runs_before = [&](int64_t p) -> int64_t {  // runs that start before sorted position p
    if (p < n) return head_scan[p];
    const bool last_head = n == 1 || keys[n - 1] != keys[n - 2] ||
                           seg_find(cs.c0, cs.n, n - 1) != seg_find(cs.c0, cs.n, n - 2);
    return (int64_t)head_scan[n - 1] + (last_head ? 1 : 0);
  };
  counts[k] = (int)(runs_before(b) - runs_before(a));
}

}  // namespace

bool make_catset(const int64_t* c0, int n_cat, CatSet& cs) {
  if (n_cat < 1 || n_cat > kMaxCatSet) return false;
  cs.n = n_cat;
  cs.c0[0] = 0;
  cs.coff[0] = 0;
  cs.tile0[0] = 0;
  cs.stile0[0] = 0;
  for (int k = 0; k < n_cat; ++k) {
    const int64_t nk = c0[k + 1] - c0[k];
    cs.c0[k + 1] = c0[k + 1] - c0[0];
    cs.coff[k + 1] = cs.coff[k] + (nk > 0 ? (int64_t)grid_cells_cap(nk) : 0);
    cs.tile0[k + 1] = cs.tile0[k] + (int)((nk + kBBoxTile - 1) / kBBoxTile);
    cs.stile0[k + 1] = cs.stile0[k] + (int)((nk + kSortTile - 1) / kSortTile);
  }
  // positions and cell-list entries stay below 2^31
  return cs.coff[n_cat] < ((int64_t)1 << 31) && cs.c0[n_cat] < ((int64_t)1 << 31) - 1;
}

cudaError_t bbox_batch(const double* pos, const CatSet& cs, double* part, double* bbox, cudaStream_t s) {
  if (cs.tile0[cs.n] > 0) {
    bbox_tiles<<<cs.tile0[cs.n], 256, 0, s>>>(pos, cs, part);
    ++g_launches;
  }
  bbox_cats<<<(cs.n + 127) / 128, 128, 0, s>>>(cs, part, bbox);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t grid_sort_batch(const double* pos, const double* shear, const double* wts, const CatSet& cs,
                            const double* bbox, double rmax, GridGeom* geoms, bool want_f32, GridBuffers& gb,
                            int** perm_out, int* status, cudaStream_t s) {
  const int64_t n = cs.c0[cs.n];
  geom_cats<<<(cs.n + 127) / 128, 128, 0, s>>>(cs, bbox, rmax, 0.0, geoms, status);
  ++g_launches;
  if (n == 0) {
    *perm_out = gb.perm;
    return cudaGetLastError();
  }
  const unsigned nblk = (unsigned)((n + 255) / 256);
  keys_cats<<<nblk, 256, 0, s>>>(pos, cs, geoms, gb.keys, gb.perm, status);
  ++g_launches;
  int* keys = nullptr;
  int* perm = nullptr;
  cudaError_t e = radix_sort_cats(gb, cs, &keys, &perm, s);
  if (e != cudaSuccess) return e;
  cell_bounds_cats<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(keys, cs, geoms, gb.cell_start);
  build_sorted_cats<<<nblk, 256, 0, s>>>(pos, shear, wts, perm, keys, cs, geoms, want_f32, gb.px, gb.py, gb.xr,
                                         gb.xi, gb.w, gb.p4, gb.s4);
  g_launches += 2;
  *perm_out = perm;
  return cudaGetLastError();
}

cudaError_t reduce_batch(const double* pos, const double* shear, const double* wts, const CatSet& cs,
                         const double* bbox, double delta, GridGeom* geoms, GridBuffers& gb, unsigned* head,
                         double* rpos, double* rshear, double* rw, int* counts, int* status, cudaStream_t s) {
  const int64_t n = cs.c0[cs.n];
  geom_cats<<<(cs.n + 127) / 128, 128, 0, s>>>(cs, bbox, 0.0, delta, geoms, status);
  ++g_launches;
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * cs.n, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const unsigned nblk = (unsigned)((n + 255) / 256);
  keys_cats<<<nblk, 256, 0, s>>>(pos, cs, geoms, gb.keys, gb.perm, status);
  ++g_launches;
  int* keys = nullptr;
  int* perm = nullptr;
  cudaError_t e = radix_sort_cats(gb, cs, &keys, &perm, s);
  if (e != cudaSuccess) return e;
  run_heads_cats<<<nblk, 256, 0, s>>>(keys, cs, head);
  e = scan_exclusive(head, (size_t)n, gb.hist, s);
  if (e != cudaSuccess) return e;
  reduce_runs_cats<<<nblk, 256, 0, s>>>(keys, perm, head, cs, pos, shear, wts, rpos, rshear, rw);
  run_counts<<<(cs.n + 127) / 128, 128, 0, s>>>(head, keys, cs, counts);
  g_launches += 3;
  return cudaGetLastError();
}

}  // namespace ext4pcf
