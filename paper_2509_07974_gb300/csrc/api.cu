// C ABI of libext4pcf: argument checking, scratch management and the per-catalogue
// pipeline  grid build -> [gather -> contraction -> correction sums] per centre wave ->
// correction application.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace ext4pcf {
cudaError_t scan_exclusive(unsigned* data, size_t n, unsigned* tmp, cudaStream_t s);
cudaError_t real_space(const double* ups, int nb, int N, int nphi, double* gamma, double* norm,
                       double* scratch_norm, double* E_scratch, cudaStream_t s);
size_t real_space_smem(int N, int nphi);
int map4_nsplit(int chunk_tri, int ntri, int n_ap);
cudaError_t map4_partials(const double* ups, const double* edges_host, int nb, int N, int nphi,
                          const double* ap_host, int n_ap, double* E_scratch, double* norm_chunk,
                          double* gam_chunk, int chunk_tri, int nsplit, double* partial, cudaStream_t s);
cudaError_t map4_finish_launch(const double* partial, int ntri, int n_ap, const double* d_xipm,
                               const double* d_tb, const double* d_area, int nb, const double* d_ap,
                               double* d_m4, double* d_eb, double* d_disc, cudaStream_t s);
int map_direct_splits(int n_ap, int sm_count, double theta, double cell);
size_t map_direct_scratch(int n_ap, int nsplit);
bool contract3_supported(int N);
size_t contract3_scratch_bytes(const Layout& L, int T);
template <typename Cx>
cudaError_t contract3_wave(const Layout& L, const Cx* rec, const Cx* xw, int T, double* ups3, double2* scratch,
                           cudaStream_t s);
cudaError_t map_direct_radius(const SortedCat& cat, const double* centres, int n_ap, double theta,
                              int nsplit, void* scratch, double* rec, double* mom, cudaStream_t s);
}  // namespace ext4pcf

namespace ext4pcf {
thread_local long long g_launches = 0;
}

using namespace ext4pcf;

namespace {

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

__global__ void mask_flags(const uint8_t* __restrict__ mask, const int* __restrict__ perm, int n,
                           unsigned* __restrict__ flag) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) flag[p] = mask ? (mask[perm[p]] != 0) : 1u;
}
// centre list: concatenated sorted positions c0 + p of the catalogue's centres
__global__ void mask_compact(const unsigned* __restrict__ flag_scan, const uint8_t* __restrict__ mask,
                             const int* __restrict__ perm, int n, int c0, int* __restrict__ centres,
                             int* __restrict__ count) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && (!mask || mask[perm[p]] != 0)) centres[flag_scan[p]] = c0 + p;
  if (p == n - 1) *count = (int)flag_scan[p] + ((!mask || mask[perm[p]] != 0) ? 1 : 0);
}
// inv[i] = sorted position of galaxy i (perm: sorted position -> galaxy)
__global__ void inverse_perm(const int* __restrict__ perm, int n, int* __restrict__ inv) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) inv[perm[p]] = p;
}
__global__ void pick_centres(const int64_t* __restrict__ idx, int64_t n, const int* __restrict__ inv,
                             int* __restrict__ centres) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) centres[j] = inv[idx[j]];
}
// a wave's records as FP64 complex pairs
template <typename R>
__global__ void records_out(const ext4pcf::cplx_t<R>* __restrict__ rec, size_t n, double2* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)rec[i].x, (double)rec[i].y);
}
// the centre lists of every catalogue of a set at once: catalogue k's centres at c0[k] on,
// in sorted order, and their count (flag_scan: exclusive scan of the centre flags)
__global__ void mask_compact_cats(const unsigned* __restrict__ flag_scan, const uint8_t* __restrict__ mask,
                                  const int* __restrict__ perm, const CatSet cs, int* __restrict__ centres,
                                  int* __restrict__ count) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cs.c0[cs.n]) return;
  int lo = 0, hi = cs.n;  // the catalogue of sorted position p
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p >= cs.c0[mid]) lo = mid; else hi = mid;
  }
  const bool f = mask[perm[p]] != 0;
  const unsigned base = flag_scan[cs.c0[lo]];
  if (f) centres[cs.c0[lo] + (flag_scan[p] - base)] = (int)p;
  if (p == cs.c0[lo + 1] - 1) count[lo] = (int)(flag_scan[p] + (f ? 1u : 0u) - base);
}
__global__ void iota(int* a, int n, int c0) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) a[p] = c0 + p;
}
// status bits: 1 a bounded device-side wait ran out, 2 non-finite positions
int status_code(int st) {
  if (st & 1) return EXT4PCF_E_TIMEOUT;
  if (st & 2) return EXT4PCF_E_INVALID_ARG;
  return EXT4PCF_OK;
}

}  // namespace

struct ext4pcf_ctx {
  ext4pcf_config cfg{};
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  std::string err;
  // inputs staged from host memory
  DBuf in_pos, in_shear, in_w, in_mask, io_ups, io_xi;
  // grid
  DBuf keys, keys_alt, perm, perm_alt, cell_start, hist, px, py, xr, xi, w, p4, s4, bbox;
  // waves
  DBuf centres, flags, rec, xw, corr, counter, ncen;
  // transforms
  DBuf t_norm, t_gam, t_E, t_part, t_small;
  // direct aperture estimator: centres, per-split sums, staged outputs
  DBuf ap_cen, ap_sums, io_rec, io_mom;
  // tensor-core contraction: work items (built once per shape) and the device status word
  DBuf tc_items, tc_xb, tc_red, tc_rowmax, status, geom;
  int tc_N = -1, tc_nb = -1;
  size_t tc_items_bytes = 0;
  cudaEvent_t ev[8] = {};
  std::vector<cudaEvent_t> tev;  // per-phase timing events of one measure call (grown on demand)
  // tree approximation: per level, the reduced catalogues (cell order, per catalogue at its
  // galaxies' offsets), their sizes, and their sorted arrays and grids (at offsets by size)
  struct Level {
    DBuf rpos, rsh, rw, cnt, px, py, xr, xi, w, p4, s4, cells, geom;
  };
  Level lv[9];
  DBuf inv, rec_idx, rec_out;  // ext4pcf_multipoles: inverse sort order, centre list, staged records
  // wave sizes chosen by the autotuner, per (precision, n_max, n_bins)
  std::map<std::tuple<int, int, int>, int> tuned;
  int64_t last_wave = 0;
};

namespace {

int fail(ext4pcf_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(ext4pcf_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? EXT4PCF_E_OOM : EXT4PCF_E_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)
// the gather's launch: a centre's record (n_bins (14 n_max + 18) complex values) that does not
// fit its shared memory next to the pair buffers is refused by gather_wave with
// cudaErrorInvalidConfiguration, reported as an unsupported size
#define GK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ == cudaErrorInvalidConfiguration)                                                         \
      return fail(ctx, EXT4PCF_E_UNSUPPORTED, "the multipole record (n_bins x n_max) does not fit "  \
                                              "the gather's shared memory");                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);                                         \
  } while (0)

int ensure(ext4pcf_ctx* ctx, DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return EXT4PCF_OK;
  if (b.p) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return fail(ctx, EXT4PCF_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    want = bytes;
  }
  b.bytes = want;
  return EXT4PCF_OK;
}

#define ENSURE(buf, bytes)                           \
  do {                                               \
    int r_ = ensure(ctx, (buf), (bytes));            \
    if (r_ != EXT4PCF_OK) return r_;                 \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// synchronise the context's stream and read (and clear) its status word; *code receives
// the status as an error code
int read_status(ext4pcf_ctx* ctx, int* code) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->status.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st != 0) CK(cudaMemsetAsync(ctx->status.p, 0, 4, ctx->stream));
  *code = status_code(st);
  if (*code == EXT4PCF_E_TIMEOUT) fail(ctx, *code, "a bounded device-side wait expired in the contraction");
  else if (*code != EXT4PCF_OK) fail(ctx, *code, "non-finite positions");
  return EXT4PCF_OK;
}

}  // namespace

extern "C" {

int ext4pcf_create(ext4pcf_ctx** out, const ext4pcf_config* cfg) {
  if (!out || !cfg) return EXT4PCF_E_INVALID_ARG;
  *out = nullptr;
  if (std::getenv("EXT4PCF_FAULT") && std::strcmp(std::getenv("EXT4PCF_FAULT"), "alloc") == 0)
    return EXT4PCF_E_OOM;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return EXT4PCF_E_UNSUPPORTED;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg->device) != cudaSuccess) return EXT4PCF_E_CUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return EXT4PCF_E_UNSUPPORTED;
  if (cfg->precision < EXT4PCF_FP64 || cfg->precision > EXT4PCF_SPLIT_F16) return EXT4PCF_E_INVALID_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return EXT4PCF_E_CUDA;
  ext4pcf_ctx* ctx = new ext4pcf_ctx;
  ctx->cfg = *cfg;
  ctx->stream = static_cast<cudaStream_t>(cfg->stream);
  ctx->sm_count = prop.multiProcessorCount;
  for (auto& e : ctx->ev) cudaEventCreate(&e);
  // the status word (bits of status_code) accumulates until a synchronising call reads it
  if (cudaMalloc(&ctx->status.p, 16) != cudaSuccess || cudaMemset(ctx->status.p, 0, 16) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->status.p) cudaFree(ctx->status.p);
    delete ctx;
    return EXT4PCF_E_OOM;
  }
  ctx->status.bytes = 16;
  *out = ctx;
  return EXT4PCF_OK;
}

int ext4pcf_destroy(ext4pcf_ctx* ctx) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  cudaSetDevice(ctx->cfg.device);
  cudaStreamSynchronize(ctx->stream);
  DBuf* all[] = {&ctx->in_pos, &ctx->in_shear, &ctx->in_w, &ctx->in_mask, &ctx->io_ups, &ctx->io_xi,
                 &ctx->keys, &ctx->keys_alt, &ctx->perm, &ctx->perm_alt, &ctx->cell_start, &ctx->hist,
                 &ctx->px, &ctx->py, &ctx->xr, &ctx->xi, &ctx->w, &ctx->p4, &ctx->s4, &ctx->bbox,
                 &ctx->centres, &ctx->flags, &ctx->rec, &ctx->xw, &ctx->corr, &ctx->counter, &ctx->ncen,
                 &ctx->t_norm, &ctx->t_gam, &ctx->t_E, &ctx->t_part, &ctx->t_small, &ctx->tc_items,
                 &ctx->tc_xb, &ctx->tc_red, &ctx->tc_rowmax, &ctx->status, &ctx->geom, &ctx->ap_cen, &ctx->ap_sums, &ctx->io_rec, &ctx->io_mom};
  for (DBuf* b : all)
    if (b->p) cudaFree(b->p);
  for (auto& L : ctx->lv)
    for (DBuf* b : {&L.rpos, &L.rsh, &L.rw, &L.cnt, &L.px, &L.py, &L.xr, &L.xi, &L.w, &L.p4, &L.s4, &L.cells, &L.geom})
      if (b->p) cudaFree(b->p);
  for (DBuf* b : {&ctx->inv, &ctx->rec_idx, &ctx->rec_out})
    if (b->p) cudaFree(b->p);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : ctx->tev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return EXT4PCF_OK;
}

const char* ext4pcf_last_error(const ext4pcf_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int ext4pcf_synchronize(ext4pcf_ctx* ctx) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  ctx->err.clear();
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = EXT4PCF_OK;
  const int r = read_status(ctx, &rc);
  return r != EXT4PCF_OK ? r : rc;
}

}  // extern "C"

namespace {
// The measure pipeline.  Records mode (rec_out non-null, one catalogue): the centres are the
// galaxies rec_centres[0 .. n_rec) (indices into the catalogue) and their multipole records
// are written to rec_out instead of being contracted.
int measure_impl(ext4pcf_ctx* ctx, const double* positions, const double* shears, const double* weights,
                 int64_t n_gal, const double* radial_bins, int n_bins, int n_max, const int64_t* cat_offsets,
                 int n_cat, const int* out_slot, int n_out, const uint8_t* centre_mask, double* upsilon,
                 double* xi_acc, ext4pcf_stats* stats, const int64_t* rec_centres, int64_t n_rec, double* rec_out) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  const bool records = rec_out != nullptr;
  ctx->err.clear();
  if (std::getenv("EXT4PCF_FAULT") && std::strcmp(std::getenv("EXT4PCF_FAULT"), "arg") == 0)
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "fault injection: argument check");
  if (n_gal < 0 || n_gal > (int64_t)2000000000) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_gal out of range");
  if (n_bins < 1 || n_bins > 32) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_bins must be in 1..32");
  if (n_max < 0 || n_max > 40) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_max must be in 0..40");
  if (!radial_bins || (!upsilon && !records)) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null radial_bins or upsilon");
  if (records && (cat_offsets || centre_mask || n_rec < 0 || (n_rec > 0 && !rec_centres)))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "multipole records: one catalogue, centres by index");
  for (int64_t i = 0; records && i < n_rec; ++i)
    if (rec_centres[i] < 0 || rec_centres[i] >= n_gal)
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "centre index out of range");
  const bool tree = ctx->cfg.tree_delta1 > 0.0 && ctx->cfg.tree_levels > 0;
  if (tree && (!(ctx->cfg.tree_rmin > 0.0) || ctx->cfg.tree_levels > 8 || !std::isfinite(ctx->cfg.tree_delta1)))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "tree approximation: 1 <= tree_levels <= 8, tree_rmin > 0");
  if (n_gal > 0 && (!positions || !shears || !weights)) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null input");
  if (!(radial_bins[0] > 0.0) || !std::isfinite(radial_bins[n_bins]))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "radial_bins[0] must be > 0 and finite");
  for (int b = 0; b < n_bins; ++b)
    if (!(radial_bins[b + 1] > radial_bins[b])) return fail(ctx, EXT4PCF_E_INVALID_ARG, "radial_bins must increase");
  if (cat_offsets) {
    if (n_cat < 1) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_cat < 1");
    if (cat_offsets[0] != 0 || cat_offsets[n_cat] != n_gal)
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "cat_offsets must span [0, n_gal]");
    for (int k = 0; k < n_cat; ++k)
      if (cat_offsets[k + 1] < cat_offsets[k]) return fail(ctx, EXT4PCF_E_INVALID_ARG, "cat_offsets decrease");
  } else {
    n_cat = 1;
  }
  if (out_slot) {
    if (n_out < 1) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_out < 1");
    for (int k = 0; k < n_cat; ++k)
      if (out_slot[k] < 0 || out_slot[k] >= n_out) return fail(ctx, EXT4PCF_E_INVALID_ARG, "out_slot out of range");
  } else {
    n_out = n_cat;
  }
  const int prec = ctx->cfg.precision;
  if (prec >= EXT4PCF_TF32 && !tc_supported(Layout::make(n_max, n_bins), prec))
    return fail(ctx, EXT4PCF_E_UNSUPPORTED, "tensor-core contraction does not support this size");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = ctx->stream;
  const bool f64 = prec == EXT4PCF_FP64;
  const Layout L = Layout::make(n_max, n_bins);
  const size_t ups_elems = (size_t)9 * (2 * n_max + 1) * (2 * n_max + 1) * n_bins * n_bins * n_bins;
  const size_t ups_bytes = ups_elems * 16;

  // ---- stage host inputs / outputs
  const size_t n = (size_t)n_gal;
  const double* d_pos = positions;
  const double* d_sh = shears;
  const double* d_w = weights;
  const uint8_t* d_mask = centre_mask;
  double* d_ups = upsilon;
  double* d_xi = xi_acc;
  const bool host_ups = !records && !is_device_ptr(upsilon);
  const bool rec_host = records && !is_device_ptr(rec_out);
  if (rec_host) ENSURE(ctx->rec_out, (size_t)std::max<int64_t>(n_rec, 1) * Layout::make(n_max, n_bins).rec * 16);
  const bool host_xi = xi_acc && !is_device_ptr(xi_acc);
  if (n > 0 && !is_device_ptr(positions)) {
    ENSURE(ctx->in_pos, n * 16);
    CK(cudaMemcpyAsync(ctx->in_pos.p, positions, n * 16, cudaMemcpyHostToDevice, s));
    d_pos = (const double*)ctx->in_pos.p;
  }
  if (n > 0 && !is_device_ptr(shears)) {
    ENSURE(ctx->in_shear, n * 16);
    CK(cudaMemcpyAsync(ctx->in_shear.p, shears, n * 16, cudaMemcpyHostToDevice, s));
    d_sh = (const double*)ctx->in_shear.p;
  }
  if (n > 0 && !is_device_ptr(weights)) {
    ENSURE(ctx->in_w, n * 8);
    CK(cudaMemcpyAsync(ctx->in_w.p, weights, n * 8, cudaMemcpyHostToDevice, s));
    d_w = (const double*)ctx->in_w.p;
  }
  if (n > 0 && centre_mask && !is_device_ptr(centre_mask)) {
    ENSURE(ctx->in_mask, n);
    CK(cudaMemcpyAsync(ctx->in_mask.p, centre_mask, n, cudaMemcpyHostToDevice, s));
    d_mask = (const uint8_t*)ctx->in_mask.p;
  }
  if (host_ups) {
    ENSURE(ctx->io_ups, ups_bytes * n_out);
    CK(cudaMemcpyAsync(ctx->io_ups.p, upsilon, ups_bytes * n_out, cudaMemcpyHostToDevice, s));
    d_ups = (double*)ctx->io_ups.p;
  }
  const size_t xi_bytes = (size_t)n_bins * 6 * 8;
  if (host_xi) {
    ENSURE(ctx->io_xi, xi_bytes * n_out);
    CK(cudaMemcpyAsync(ctx->io_xi.p, xi_acc, xi_bytes * n_out, cudaMemcpyHostToDevice, s));
    d_xi = (double*)ctx->io_xi.p;
  }

  Bins bins;
  bins.nb = n_bins;
  for (int b = 0; b <= n_bins; ++b) {
    bins.e2[b] = radial_bins[b] * radial_bins[b];
    bins.e2f[b] = (float)bins.e2[b];
  }
  bins.rmax = radial_bins[n_bins];

  const bool timing = stats != nullptr;
  const long long launches0 = g_launches;
  float ms_grid = 0, ms_gather = 0, ms_contract = 0, ms_correct = 0, ms_total = 0;
  int64_t tot_centres = 0, tot_waves = 0;
  if (timing) CK(cudaEventRecord(ctx->ev[0], s));
  // phase timing without host synchronisation: events are recorded on the stream and their
  // intervals summed once at the end of the call (kind 0 grid, 1 gather, 2 contraction,
  // 3 corrections)
  struct Mark { int kind, a, b; };
  std::vector<Mark> marks;
  int nev = 0;
  auto tmark = [&]() -> int {
    if (nev >= (int)ctx->tev.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      ctx->tev.push_back(e);
    }
    if (cudaEventRecord(ctx->tev[nev], s) != cudaSuccess) return -1;
    return nev++;
  };
  int t_grid0 = -1;
  ENSURE(ctx->counter, 16);
  CK(cudaMemsetAsync(ctx->counter.p, 0, 8, s));
  const bool tc = prec == EXT4PCF_TF32 || prec == EXT4PCF_SPLIT_BF16 || prec == EXT4PCF_3XTF32 ||
                  prec == EXT4PCF_SPLIT_F16;
  // waves that pack the centres of several catalogues: the split-FP16 contraction, the gather
  // and the correction sums take segments; the other contraction forms one catalogue a wave
  const bool multi = prec == EXT4PCF_SPLIT_F16;
  if (tc) {
    if (ctx->tc_N != n_max || ctx->tc_nb != n_bins) {
      std::vector<int4> items;
      if (!tc_build_items(L, items)) return fail(ctx, EXT4PCF_E_UNSUPPORTED, "no symmetry map for the contraction table");
      ENSURE(ctx->tc_items, items.size() * sizeof(int4));
      CK(cudaMemcpy(ctx->tc_items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
      ctx->tc_items_bytes = items.size() * sizeof(int4);
      ctx->tc_N = n_max;
      ctx->tc_nb = n_bins;
    }
  }
  const long long timeout = ctx->cfg.timeout_cycles > 0 ? ctx->cfg.timeout_cycles : 20000000000LL;

  // ---- per catalogue: first galaxy, galaxy count and (when known on the host) centre count
  std::vector<int64_t> c0v(n_cat + 1, 0);
  for (int k = 0; k < n_cat; ++k) c0v[k + 1] = cat_offsets ? cat_offsets[k + 1] : n_gal;
  std::vector<int64_t> ncent(n_cat, -1);  // -1: counted on the device (a device-resident mask)
  const bool host_mask = centre_mask && !is_device_ptr(centre_mask);
  for (int k = 0; k < n_cat; ++k) {
    const int64_t nk = c0v[k + 1] - c0v[k];
    if (records) {
      ncent[k] = n_rec;
    } else if (!centre_mask) {
      ncent[k] = nk;
    } else if (host_mask) {
      int64_t c = 0;
      for (int64_t i = c0v[k]; i < c0v[k + 1]; ++i) c += centre_mask[i] != 0;
      ncent[k] = c;
    }
  }
  int64_t nk_max = 0, cells_total = 0;
  std::vector<int64_t> cell_off(n_cat + 1, 0);
  for (int k = 0; k < n_cat; ++k) {
    const int64_t nk = c0v[k + 1] - c0v[k];
    nk_max = std::max(nk_max, nk);
    cell_off[k + 1] = cell_off[k] + (nk > 0 ? (int64_t)grid_cells_cap(nk) : 0);
  }
  cells_total = cell_off[n_cat];

  // ---- grids of all catalogues (device geometry, no host round trip), into the concatenated
  // sorted arrays; centre lists hold concatenated positions
  // one batched build of every catalogue's grid when they fit one set (kMaxCatSet
  // catalogues), else one build per catalogue; the two give the same arrays
  CatSet cset;
  const bool batched = make_catset(c0v.data(), n_cat, cset);
  const int64_t nsort = batched ? (int64_t)n : nk_max;  // keys sorted at once
  ENSURE(ctx->ncen, (size_t)(n_cat + 1) * sizeof(int));
  ENSURE(ctx->bbox, batched ? ((size_t)4 * n_cat + 4 * (size_t)cset.tile0[n_cat] + 4) * 8 : (4 + 4 * 512) * 8);
  ENSURE(ctx->geom, (size_t)std::max(n_cat, 1) * sizeof(GridGeom));
  ENSURE(ctx->cell_start, (size_t)std::max<int64_t>(cells_total, 1) * 4);
  if (centre_mask) CK(cudaMemsetAsync(ctx->ncen.p, 0, (size_t)(n_cat + 1) * sizeof(int), s));
  {
    // sort tiles: a batched sort's tiles never span two catalogues (at most one partial
    // tile per catalogue more than one array needs)
    const size_t ntiles = (size_t)((nsort + 2047) / 2048) + (size_t)n_cat + 1;
    ENSURE(ctx->keys, (size_t)nsort * 4); ENSURE(ctx->keys_alt, (size_t)nsort * 4);
    ENSURE(ctx->perm, (size_t)nsort * 4); ENSURE(ctx->perm_alt, (size_t)nsort * 4);
    ENSURE(ctx->hist, ((size_t)256 * ntiles * 2 + 4096) * 4);
    ENSURE(ctx->px, n * 8); ENSURE(ctx->py, n * 8);
    ENSURE(ctx->xr, n * 8); ENSURE(ctx->xi, n * 8); ENSURE(ctx->w, n * 8);
    if (!f64) { ENSURE(ctx->p4, n * 16); ENSURE(ctx->s4, n * 16); }
    ENSURE(ctx->centres, n * 4);
    if (centre_mask || tree) ENSURE(ctx->flags, ((size_t)nsort + (size_t)nsort / 1000 + 4096) * 4);
  }
  double* cat_bbox = (double*)ctx->bbox.p;        // batched: [n_cat][4], then the tiles' partials
  double* bbox_part = cat_bbox + 4 * (size_t)n_cat;
  SortedCat cat{};
  cat.n = (int)n;
  cat.px = (const double*)ctx->px.p; cat.py = (const double*)ctx->py.p;
  cat.xr = (const double*)ctx->xr.p; cat.xi = (const double*)ctx->xi.p; cat.w = (const double*)ctx->w.p;
  cat.p4 = (const float4*)ctx->p4.p; cat.s4 = (const float4*)ctx->s4.p;
  GridGeom* geoms = (GridGeom*)ctx->geom.p;
  int* cells = (int*)ctx->cell_start.p;
  int* clist = (int*)ctx->centres.p;
  int* ncen_d = (int*)ctx->ncen.p;
  if (timing) t_grid0 = tmark();
  if (batched) {
    GridBuffers gb{};
    gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
    gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
    gb.cell_start = cells; gb.cell_cap = (size_t)cells_total;
    gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
    gb.px = (double*)ctx->px.p; gb.py = (double*)ctx->py.p;
    gb.xr = (double*)ctx->xr.p; gb.xi = (double*)ctx->xi.p; gb.w = (double*)ctx->w.p;
    gb.p4 = f64 ? nullptr : (float4*)ctx->p4.p; gb.s4 = f64 ? nullptr : (float4*)ctx->s4.p;
    CK(bbox_batch(d_pos, cset, bbox_part, cat_bbox, s));
    int* perm = nullptr;
    CK(grid_sort_batch(d_pos, d_sh, d_w, cset, cat_bbox, bins.rmax, geoms, !f64, gb, &perm, (int*)ctx->status.p, s));
    const int nn = (int)n;
    if (nn == 0) {
      // no galaxies: no centres (the counts were cleared above)
    } else if (records) {  // one catalogue: the requested galaxies, through the inverse of the sort order
      ENSURE(ctx->inv, (size_t)nn * 4);
      ENSURE(ctx->rec_idx, (size_t)std::max<int64_t>(n_rec, 1) * 8);
      inverse_perm<<<(nn + 255) / 256, 256, 0, s>>>(perm, nn, (int*)ctx->inv.p);
      if (n_rec > 0) {
        CK(cudaMemcpyAsync(ctx->rec_idx.p, rec_centres, (size_t)n_rec * 8, cudaMemcpyHostToDevice, s));
        pick_centres<<<(int)((n_rec + 255) / 256), 256, 0, s>>>((const int64_t*)ctx->rec_idx.p, n_rec,
                                                               (const int*)ctx->inv.p, clist);
      }
      g_launches += 2;
      CK(cudaGetLastError());
    } else if (d_mask) {  // every catalogue's centre list and count at once
      unsigned* flag = (unsigned*)ctx->flags.p;
      mask_flags<<<(nn + 255) / 256, 256, 0, s>>>(d_mask, perm, nn, flag);
      CK(scan_exclusive(flag, (size_t)nn, (unsigned*)ctx->hist.p, s));
      mask_compact_cats<<<(nn + 255) / 256, 256, 0, s>>>(flag, d_mask, perm, cset, clist, ncen_d);
      g_launches += 2;
      CK(cudaGetLastError());
    } else {
      iota<<<(nn + 255) / 256, 256, 0, s>>>(clist, nn, 0);
      ++g_launches;
      CK(cudaGetLastError());
    }
  }
  for (int k = 0; k < n_cat && !batched; ++k) {
    const int64_t c0 = c0v[k];
    const int nk = (int)(c0v[k + 1] - c0);
    if (nk == 0) continue;
    const uint8_t* mask_k = d_mask ? d_mask + c0 : nullptr;
    CK(grid_bbox(d_pos + 2 * c0, nk, (double*)ctx->bbox.p, s));
    GridBuffers gb;
    gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
    gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
    gb.cell_start = cells + cell_off[k]; gb.cell_cap = (size_t)(cell_off[k + 1] - cell_off[k]);
    gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
    gb.px = (double*)ctx->px.p + c0; gb.py = (double*)ctx->py.p + c0;
    gb.xr = (double*)ctx->xr.p + c0; gb.xi = (double*)ctx->xi.p + c0; gb.w = (double*)ctx->w.p + c0;
    gb.p4 = f64 ? nullptr : (float4*)ctx->p4.p + c0; gb.s4 = f64 ? nullptr : (float4*)ctx->s4.p + c0;
    gb.bbox = (double*)ctx->bbox.p;
    SortedCat sk;
    CK(grid_sort_device(d_pos + 2 * c0, d_sh + 2 * c0, d_w + c0, nk, (int)c0, (const double*)ctx->bbox.p,
                        bins.rmax, geoms + k, !f64, gb, sk, (int*)ctx->status.p, s));
    // centre list (concatenated sorted positions of the centres); with a mask the count goes
    // to ncen[k] on the device
    if (records) {  // the requested galaxies, through the inverse of the sort order
      ENSURE(ctx->inv, (size_t)nk * 4);
      ENSURE(ctx->rec_idx, (size_t)std::max<int64_t>(n_rec, 1) * 8);
      inverse_perm<<<(nk + 255) / 256, 256, 0, s>>>(sk.perm, nk, (int*)ctx->inv.p);
      if (n_rec > 0) {
        CK(cudaMemcpyAsync(ctx->rec_idx.p, rec_centres, (size_t)n_rec * 8, cudaMemcpyHostToDevice, s));
        pick_centres<<<(int)((n_rec + 255) / 256), 256, 0, s>>>((const int64_t*)ctx->rec_idx.p, n_rec,
                                                               (const int*)ctx->inv.p, clist);
      }
      g_launches += 2;
      CK(cudaGetLastError());
    } else if (mask_k) {
      unsigned* flag = (unsigned*)ctx->flags.p;
      mask_flags<<<(nk + 255) / 256, 256, 0, s>>>(mask_k, sk.perm, nk, flag);
      g_launches += 2;  // flags + compaction
      unsigned* tmp = (unsigned*)ctx->hist.p;  // reuse as scan scratch
      CK(scan_exclusive(flag, (size_t)nk, tmp, s));
      mask_compact<<<(nk + 255) / 256, 256, 0, s>>>(flag, mask_k, sk.perm, nk, (int)c0, clist + c0, ncen_d + k);
      CK(cudaGetLastError());
    } else {
      iota<<<(nk + 255) / 256, 256, 0, s>>>(clist + c0, nk, (int)c0);
      ++g_launches;
      CK(cudaGetLastError());
    }
  }
  // ---- tree approximation: the level of every radial bin (the coarsest d with
  // Theta_lo / Delta_d >= r_min, else 0: the galaxies), the reduced catalogues of the levels in
  // use and their grids; the gather then runs one pass per level over that level's bins
  struct Pass {
    int level, blo, bhi;
    SortedCat cat;
    const GridGeom* geoms;
    const int* cells;
    std::vector<int64_t> coff;
    Bins bins;
  };
  std::vector<Pass> passes;
  {
    std::vector<int> blev(n_bins, 0);
    if (tree)
      for (int b = 0; b < n_bins; ++b)
        for (int d = ctx->cfg.tree_levels; d >= 1; --d)
          if (radial_bins[b] / (ctx->cfg.tree_delta1 * std::ldexp(1.0, d - 1)) >= ctx->cfg.tree_rmin) {
            blev[b] = d;
            break;
          }
    for (int b = 0; b < n_bins;) {  // levels never decrease with the bin (its inner edge grows)
      int e = b;
      while (e < n_bins && blev[e] == blev[b]) ++e;
      Pass P;
      P.level = blev[b];
      P.blo = b;
      P.bhi = e;
      P.bins = bins;
      for (int q = 0; q <= n_bins; ++q) {  // bins outside [blo, bhi) get zero width
        const int qq = q < b ? b : (q > e ? e : q);
        P.bins.e2[q] = bins.e2[qq];
        P.bins.e2f[q] = bins.e2f[qq];
      }
      P.bins.rmax = radial_bins[e];
      passes.push_back(P);
      b = e;
    }
  }
  for (Pass& P : passes)
    if (P.level == 0) {
      P.cat = cat;
      P.geoms = geoms;
      P.cells = cells;
      P.coff = cell_off;
    }
  if (tree) {
    // reduced catalogues, per level in use and catalogue, at the galaxies' offsets
    std::vector<int> lev_used;
    for (const Pass& P : passes)
      if (P.level > 0) lev_used.push_back(P.level);
    ENSURE(ctx->flags, ((size_t)nk_max + (size_t)nk_max / 1000 + 4096) * 4);
    for (int d : lev_used) {
      ext4pcf_ctx::Level& V = ctx->lv[d];
      ENSURE(V.rpos, n * 16); ENSURE(V.rsh, n * 16); ENSURE(V.rw, n * 8);
      ENSURE(V.cnt, (size_t)(n_cat + 1) * 4); ENSURE(V.geom, (size_t)std::max(n_cat, 1) * sizeof(GridGeom));
      const double delta = ctx->cfg.tree_delta1 * std::ldexp(1.0, d - 1);
      if (batched) {  // every catalogue at once, concatenated in catalogue order
        GridBuffers gb{};
        gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
        gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
        gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
        CK(reduce_batch(d_pos, d_sh, d_w, cset, cat_bbox, delta, (GridGeom*)V.geom.p, gb, (unsigned*)ctx->flags.p,
                        (double*)V.rpos.p, (double*)V.rsh.p, (double*)V.rw.p, (int*)V.cnt.p, (int*)ctx->status.p,
                        s));
      }
      for (int k = 0; k < n_cat && !batched; ++k) {
        const int64_t c0 = c0v[k];
        const int nk = (int)(c0v[k + 1] - c0);
        GridBuffers gb{};
        gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
        gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
        gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
        CK(grid_bbox(d_pos + 2 * c0, nk, (double*)ctx->bbox.p, s));
        CK(reduce_catalogue(d_pos + 2 * c0, d_sh + 2 * c0, d_w + c0, nk, (const double*)ctx->bbox.p, delta,
                            (GridGeom*)V.geom.p + k, gb, (unsigned*)ctx->flags.p, (double*)V.rpos.p + 2 * c0,
                            (double*)V.rsh.p + 2 * c0, (double*)V.rw.p + c0, (int*)V.cnt.p + k,
                            (int*)ctx->status.p, s));
      }
    }
    // their sizes (the one synchronisation of the tree approximation)
    std::vector<std::vector<int>> m(9, std::vector<int>(n_cat, 0));
    for (int d : lev_used) CK(cudaMemcpyAsync(m[d].data(), ctx->lv[d].cnt.p, (size_t)n_cat * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (Pass& P : passes) {
      if (P.level == 0) continue;
      const int d = P.level;
      ext4pcf_ctx::Level& V = ctx->lv[d];
      std::vector<int64_t> cm(n_cat + 1, 0);
      P.coff.assign(n_cat + 1, 0);
      for (int k = 0; k < n_cat; ++k) {
        cm[k + 1] = cm[k] + m[d][k];
        P.coff[k + 1] = P.coff[k] + (m[d][k] > 0 ? (int64_t)grid_cells_cap(m[d][k]) : 0);
      }
      const size_t nm = (size_t)std::max<int64_t>(cm[n_cat], 1);
      ENSURE(V.px, nm * 8); ENSURE(V.py, nm * 8); ENSURE(V.xr, nm * 8); ENSURE(V.xi, nm * 8); ENSURE(V.w, nm * 8);
      if (!f64) { ENSURE(V.p4, nm * 16); ENSURE(V.s4, nm * 16); }
      ENSURE(V.cells, (size_t)std::max<int64_t>(P.coff[n_cat], 1) * 4);
      CatSet csr;
      if (batched && !make_catset(cm.data(), n_cat, csr))  // (fewer galaxies and cells than the set's)
        return fail(ctx, EXT4PCF_E_UNSUPPORTED, "reduced catalogues beyond one set");
      if (batched) {  // the reduced catalogues are concatenated
        GridBuffers gb{};
        gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
        gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
        gb.cell_start = (int*)V.cells.p; gb.cell_cap = (size_t)P.coff[n_cat];
        gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
        gb.px = (double*)V.px.p; gb.py = (double*)V.py.p;
        gb.xr = (double*)V.xr.p; gb.xi = (double*)V.xi.p; gb.w = (double*)V.w.p;
        gb.p4 = f64 ? nullptr : (float4*)V.p4.p; gb.s4 = f64 ? nullptr : (float4*)V.s4.p;
        const double* rp = (const double*)V.rpos.p;
        CK(bbox_batch(rp, csr, bbox_part, cat_bbox, s));  // the galaxies' boxes are no longer needed
        int* perm = nullptr;
        CK(grid_sort_batch(rp, (const double*)V.rsh.p, (const double*)V.rw.p, csr, cat_bbox, P.bins.rmax,
                           (GridGeom*)V.geom.p, !f64, gb, &perm, (int*)ctx->status.p, s));
      }
      for (int k = 0; k < n_cat && !batched; ++k) {
        const int mk = m[d][k];
        if (mk == 0) continue;
        const int64_t c0 = c0v[k];
        GridBuffers gb{};
        gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
        gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
        gb.cell_start = (int*)V.cells.p + P.coff[k]; gb.cell_cap = (size_t)(P.coff[k + 1] - P.coff[k]);
        gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
        gb.px = (double*)V.px.p + cm[k]; gb.py = (double*)V.py.p + cm[k];
        gb.xr = (double*)V.xr.p + cm[k]; gb.xi = (double*)V.xi.p + cm[k]; gb.w = (double*)V.w.p + cm[k];
        gb.p4 = f64 ? nullptr : (float4*)V.p4.p + cm[k]; gb.s4 = f64 ? nullptr : (float4*)V.s4.p + cm[k];
        gb.bbox = (double*)ctx->bbox.p;
        SortedCat sk;
        const double* rp = (const double*)V.rpos.p + 2 * c0;
        CK(grid_bbox(rp, mk, (double*)ctx->bbox.p, s));
        CK(grid_sort_device(rp, (const double*)V.rsh.p + 2 * c0, (const double*)V.rw.p + c0, mk, (int)cm[k],
                            (const double*)ctx->bbox.p, P.bins.rmax, (GridGeom*)V.geom.p + k, !f64, gb, sk,
                            (int*)ctx->status.p, s));
      }
      P.cat = SortedCat{};
      P.cat.n = (int)cm[n_cat];
      P.cat.px = (const double*)V.px.p; P.cat.py = (const double*)V.py.p;
      P.cat.xr = (const double*)V.xr.p; P.cat.xi = (const double*)V.xi.p; P.cat.w = (const double*)V.w.p;
      P.cat.p4 = (const float4*)V.p4.p; P.cat.s4 = (const float4*)V.s4.p;
      P.geoms = (const GridGeom*)V.geom.p;
      P.cells = (const int*)V.cells.p;
    }
  }
  if (timing) marks.push_back({0, t_grid0, tmark()});
  for (int k = 0; k < n_cat; ++k)
    if (ncent[k] >= 0) tot_centres += ncent[k];

  // ---- waves.  Size from the configuration, else the autotuner's choice for this shape, else
  // the default; capped so that the per-wave scratch fits ext4pcf_config.workspace_bytes
  const size_t cbytes = f64 ? sizeof(double2) : sizeof(float2);
  auto wave_bytes = [&](int t) -> size_t {
    size_t b = (size_t)t * L.rec * cbytes + (size_t)t * 2 * cbytes;
    if (tc) b += contract_tc_xb_bytes(L, t, prec);
    return b;
  };
  const auto key = std::make_tuple(prec, n_max, n_bins);
  const auto tit = ctx->tuned.find(key);
  int T = ctx->cfg.wave_centres > 0 ? ctx->cfg.wave_centres
          : tit != ctx->tuned.end()  ? tit->second
                                     : (f64 ? 4096 : 8192);
  const size_t cap = ctx->cfg.workspace_bytes > 0 ? (size_t)ctx->cfg.workspace_bytes : (size_t)-1;
  while (T > 32 && wave_bytes(T) > cap) T /= 2;
  if (wave_bytes(T) > cap) return fail(ctx, EXT4PCF_E_OOM, "workspace_bytes too small for a wave of 32 centres");
  // records a wave can need: every centre list padded to a multiple of 64
  int64_t list_total = 0, known_total = 0;
  bool all_known = true;
  for (int k = 0; k < n_cat; ++k) {
    const int64_t len = ncent[k] >= 0 ? ncent[k] : c0v[k + 1] - c0v[k];
    list_total += (len + 63) / 64 * 64;
    if (ncent[k] < 0) all_known = false;
    else known_total += ncent[k];
  }
  // autotuning (first call of a shape, centre counts known on the host, enough centres): the
  // first waves take the candidate sizes in turn -- real waves of the result, so no work is
  // repeated -- and are timed; the fastest per centre is kept for this shape.  These waves
  // synchronise.
  std::vector<int> trial;
  if (ctx->cfg.autotune && ctx->cfg.wave_centres <= 0 && tit == ctx->tuned.end() && all_known && !records) {
    const int cand[4] = {2048, 4096, 8192, 16384};
    int64_t need = 0;
    for (int c : cand)
      if (wave_bytes(c) <= cap) {
        trial.push_back(c);
        need += c;
      }
    if (trial.empty() || need > known_total) trial.clear();
  }
  int Tmax = T;
  for (int c : trial) Tmax = std::max(Tmax, c);
  if ((int64_t)Tmax > list_total) Tmax = (int)std::max<int64_t>(list_total, 1);
  if ((int64_t)T > list_total) T = (int)std::max<int64_t>(list_total, 1);
  if (Tmax < T) Tmax = T;
  ENSURE(ctx->rec, (size_t)Tmax * L.rec * cbytes);
  if (tc) {
    ENSURE(ctx->tc_xb, contract_tc_xb_bytes(L, Tmax, prec));
    if (prec == EXT4PCF_SPLIT_F16) ENSURE(ctx->tc_rowmax, contract_h16_rowmax_bytes(L));
  }
  ENSURE(ctx->xw, (size_t)Tmax * 2 * cbytes);
  std::vector<float> trial_ms;
  const size_t corr_doubles = corrections_size(L);
  ENSURE(ctx->corr, corr_doubles * 8 * n_out);
  CK(cudaMemsetAsync(ctx->corr.p, 0, corr_doubles * 8 * n_out, s));
  const size_t red_doubles = tc ? tc_reduced_doubles(L) : 0;
  if (tc) {
    ENSURE(ctx->tc_red, red_doubles * 8 * n_out);
    CK(cudaMemsetAsync(ctx->tc_red.p, 0, red_doubles * 8 * n_out, s));
  }
  // Wave planner: the catalogues' centre lists in order.  With `multi`, a wave packs runs of
  // several lists whose lengths are known on the host, each starting at a multiple of 64
  // records; otherwise (or for a list counted on the device) a wave is one run of one list.
  int pk = 0;
  int64_t pw0 = 0;
  auto slot_of = [&](int k) { return out_slot ? out_slot[k] : k; };
  auto next_plan = [&](int Tg, WavePlan& P) -> bool {
    P.nseg = 0;
    P.total = 0;
    int fill = 0;
    while (pk < n_cat) {
      const int64_t cnt = ncent[pk];
      const int64_t len = cnt >= 0 ? cnt : c0v[pk + 1] - c0v[pk];
      if (pw0 >= len) {
        ++pk;
        pw0 = 0;
        continue;
      }
      const bool single = !multi || cnt < 0;
      if (single && P.nseg > 0) break;
      const int space = Tg - fill;
      if (space <= 0) break;
      const int take = (int)std::min<int64_t>(len - pw0, space);
      WaveSeg& g = P.seg[P.nseg++];
      g.centres = clist + c0v[pk];
      g.n_live = cnt >= 0 ? nullptr : ncen_d + pk;
      g.geom = geoms + pk;
      g.cell_start = cells + cell_off[pk];
      g.w0 = (int)pw0;
      g.t = take;
      g.off = fill;
      g.slot = slot_of(pk);
      g.cat = pk;
      P.total = fill + take;
      pw0 += take;
      fill = (fill + take + 63) / 64 * 64;
      if (single || fill >= Tg || P.nseg == kMaxSegs) break;
    }
    return P.nseg > 0;
  };
  int t_w0 = -1, t_w1 = -1, t_w2 = -1;
  int largest_wave = 0;
  size_t wave_i = 0;
  WavePlan P;
  double* red_base = (double*)ctx->tc_red.p;
  double* corr_base = (double*)ctx->corr.p;
  for (;;) {
    const bool tuning = wave_i < trial.size();
    if (!next_plan(tuning ? trial[wave_i] : T, P)) break;
    const WaveSeg& g0 = P.seg[0];  // the one segment of a one-catalogue wave
    largest_wave = std::max(largest_wave, P.total);
    if (tuning) CK(cudaEventRecord(ctx->ev[1], s));
    if (timing) t_w0 = tmark();
    for (size_t pi = 0; pi < passes.size(); ++pi) {  // one pass per level: its bins, its neighbours
      const Pass& G = passes[pi];
      WavePlan Q = P;
      for (int q = 0; q < Q.nseg; ++q) {
        Q.seg[q].geom = G.geoms + Q.seg[q].cat;
        Q.seg[q].cell_start = G.cells + G.coff[Q.seg[q].cat];
      }
      if (f64) {
        GK(gather_wave<double>(G.cat, cat, G.bins, L, Q, pi > 0, (double2*)ctx->rec.p, (double2*)ctx->xw.p,
                               (unsigned long long*)ctx->counter.p, ctx->sm_count, s));
      } else {
        GK(gather_wave<float>(G.cat, cat, G.bins, L, Q, pi > 0, (float2*)ctx->rec.p, (float2*)ctx->xw.p,
                              (unsigned long long*)ctx->counter.p, ctx->sm_count, s));
      }
    }
    if (records) {  // the wave's records to the output, at the centres' places in the request
      const size_t nrec = (size_t)g0.t * L.rec;
      double2* dst = (double2*)(rec_host ? ctx->rec_out.p : (void*)rec_out) + (size_t)g0.w0 * L.rec;
      if (f64) records_out<double><<<1024, 256, 0, s>>>((const double2*)ctx->rec.p, nrec, dst);
      else records_out<float><<<1024, 256, 0, s>>>((const float2*)ctx->rec.p, nrec, dst);
      ++g_launches;
      CK(cudaGetLastError());
      ++wave_i;
      ++tot_waves;
      continue;
    }
    if (timing) t_w1 = tmark();
    if (f64) {
      CK(contract_wave<double>(L, (const double2*)ctx->rec.p, (const double2*)ctx->xw.p, g0.t, g0.n_live, g0.w0,
                               d_ups + 2 * ups_elems * (size_t)g0.slot, s));
    } else if (prec == EXT4PCF_FP32) {
      CK(contract_wave<float>(L, (const float2*)ctx->rec.p, (const float2*)ctx->xw.p, g0.t, g0.n_live, g0.w0,
                              d_ups + 2 * ups_elems * (size_t)g0.slot, s));
    } else if (prec == EXT4PCF_SPLIT_F16) {
      CK(contract_wave_h16(L, (const float2*)ctx->rec.p, (const float2*)ctx->xw.p, P, red_base,
                           (const int4*)ctx->tc_items.p, (int)(ctx->tc_items_bytes / sizeof(int4)),
                           (float2*)ctx->tc_xb.p, (unsigned*)ctx->tc_rowmax.p, (int*)ctx->status.p, timeout, s));
    } else {
      CK(contract_wave_tc(L, (const float2*)ctx->rec.p, (const float2*)ctx->xw.p, g0.t, g0.n_live, g0.w0,
                          red_base + red_doubles * (size_t)g0.slot, prec, (const int4*)ctx->tc_items.p,
                          (int)(ctx->tc_items_bytes / sizeof(int4)), (float2*)ctx->tc_xb.p,
                          (unsigned*)ctx->tc_rowmax.p, (int*)ctx->status.p, timeout, s));
    }
    if (timing) t_w2 = tmark();
    if (f64) {
      CK(corrections_wave<double>(L, (const double2*)ctx->rec.p, (const double2*)ctx->xw.p, P, corr_base, d_xi, s));
    } else {
      CK(corrections_wave<float>(L, (const float2*)ctx->rec.p, (const float2*)ctx->xw.p, P, corr_base, d_xi, s));
    }
    if (timing) {
      const int t_w3 = tmark();
      marks.push_back({1, t_w0, t_w1});
      marks.push_back({2, t_w1, t_w2});
      marks.push_back({3, t_w2, t_w3});
    }
    if (tuning) {
      float ms = 0.f;
      CK(cudaEventRecord(ctx->ev[2], s));
      CK(cudaEventSynchronize(ctx->ev[2]));
      CK(cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]));
      trial_ms.push_back(ms / (float)std::max(1, P.total));
      if (trial_ms.size() == trial.size()) {
        size_t best = 0;
        for (size_t i = 1; i < trial.size(); ++i)
          if (trial_ms[i] < trial_ms[best]) best = i;
        T = trial[best];
        ctx->tuned[key] = T;
      }
    }
    ++wave_i;
    ++tot_waves;
  }
  ctx->last_wave = std::min(T, largest_wave);  // the wave size in use (trial waves aside)
  if (records && rec_host && n_rec > 0)
    CK(cudaMemcpyAsync(rec_out, ctx->rec_out.p, (size_t)n_rec * L.rec * 16, cudaMemcpyDeviceToHost, s));
  // ---- per output slot: every ordered triple from the reduced array, then the corrections
  for (int o = 0; o < n_out && !records; ++o) {
    double* ups_o = d_ups + 2 * ups_elems * (size_t)o;
    if (tc) CK(tc_expand(L, red_base + red_doubles * (size_t)o, ups_o, s));
    CK(corrections_apply(L, corr_base + corr_doubles * (size_t)o, ups_o, s));
  }
  if (host_ups) CK(cudaMemcpyAsync(upsilon, d_ups, ups_bytes * n_out, cudaMemcpyDeviceToHost, s));
  if (host_xi) CK(cudaMemcpyAsync(xi_acc, d_xi, xi_bytes * n_out, cudaMemcpyDeviceToHost, s));
  // a call that synchronises anyway (host outputs or statistics) reports the status word;
  // a device-only call returns after enqueueing and leaves it to ext4pcf_synchronize
  if (host_ups || host_xi || timing || rec_host) {
    int rc = EXT4PCF_OK;
    const int r = read_status(ctx, &rc);
    if (r != EXT4PCF_OK) return r;
    if (rc != EXT4PCF_OK) return rc;
  }
  if (timing) {
    unsigned long long pairs = 0;
    CK(cudaMemcpyAsync(&pairs, ctx->counter.p, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev[7], s));
    CK(cudaEventSynchronize(ctx->ev[7]));
    cudaEventElapsedTime(&ms_total, ctx->ev[0], ctx->ev[7]);
    for (const Mark& m : marks) {
      float t = 0.f;
      if (m.a < 0 || m.b < 0 || cudaEventElapsedTime(&t, ctx->tev[m.a], ctx->tev[m.b]) != cudaSuccess) continue;
      if (m.kind == 0) ms_grid += t;
      else if (m.kind == 1) ms_gather += t;
      else if (m.kind == 2) ms_contract += t;
      else ms_correct += t;
    }
    if (centre_mask && !host_mask) {  // counts that only the device knows
      std::vector<int> nc(n_cat);
      CK(cudaMemcpyAsync(nc.data(), ctx->ncen.p, (size_t)n_cat * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int k = 0; k < n_cat; ++k)
        if (ncent[k] < 0) tot_centres += nc[k];
    }
    stats->pairs = (int64_t)pairs;
    stats->centres = tot_centres;
    stats->wave_centres = ctx->last_wave;
    stats->waves = tot_waves;
    stats->launches = (int64_t)(g_launches - launches0);
    stats->ms_grid = ms_grid;
    stats->ms_gather = ms_gather;
    stats->ms_contract = ms_contract;
    stats->ms_correct = ms_correct;
    stats->ms_total = ms_total;
  }
  CK(cudaGetLastError());
  return EXT4PCF_OK;
}
}  // namespace

extern "C" {

int ext4pcf_measure_batch(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                          const double* weights, int64_t n_gal, const double* radial_bins, int n_bins,
                          int n_max, const int64_t* cat_offsets, int n_cat, const int* out_slot, int n_out,
                          const uint8_t* centre_mask, double* upsilon, double* xi_acc, ext4pcf_stats* stats) {
  return measure_impl(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max, cat_offsets, n_cat,
                      out_slot, n_out, centre_mask, upsilon, xi_acc, stats, nullptr, 0, nullptr);
}

int ext4pcf_measure(ext4pcf_ctx* ctx, const double* positions, const double* shears,
                    const double* weights, int64_t n_gal, const double* radial_bins, int n_bins,
                    int n_max, const int64_t* cat_offsets, int n_cat, const uint8_t* centre_mask,
                    double* upsilon, double* xi_acc, ext4pcf_stats* stats) {
  return measure_impl(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max, cat_offsets, n_cat,
                      nullptr, 0, centre_mask, upsilon, xi_acc, stats, nullptr, 0, nullptr);
}

int ext4pcf_multipoles(ext4pcf_ctx* ctx, const double* positions, const double* shears, const double* weights,
                       int64_t n_gal, const double* radial_bins, int n_bins, int n_max, const int64_t* centres,
                       int64_t n_centres, double* records) {
  if (!records) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null records");
  return measure_impl(ctx, positions, shears, weights, n_gal, radial_bins, n_bins, n_max, nullptr, 1, nullptr, 0,
                      nullptr, nullptr, nullptr, nullptr, centres, n_centres, records);
}

int ext4pcf_to_real_space(ext4pcf_ctx* ctx, const double* upsilon, int n_bins, int n_max, int n_phi,
                          double* gamma, double* norm) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  ctx->err.clear();
  if (!upsilon || !gamma || !norm) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null pointer");
  if (n_bins < 1 || n_bins > 32 || n_max < 0 || n_max > 40 || n_phi < 1 || n_phi > 1024)
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "sizes out of range");
  if (!is_device_ptr(upsilon) || !is_device_ptr(gamma) || !is_device_ptr(norm))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "to_real_space takes device pointers");
  if (real_space_smem(n_max, n_phi) > 227 * 1024) return fail(ctx, EXT4PCF_E_UNSUPPORTED, "n_max * n_phi too large");
  CK(cudaSetDevice(ctx->cfg.device));
  const size_t ntri = (size_t)n_bins * n_bins * n_bins;
  ENSURE(ctx->t_norm, ntri * n_phi * n_phi * 8);
  ENSURE(ctx->t_E, (size_t)(2 * n_max + 1) * n_phi * 16);
  CK(real_space(upsilon, n_bins, n_max, n_phi, gamma, norm, (double*)ctx->t_norm.p, (double*)ctx->t_E.p,
                ctx->stream));
  return EXT4PCF_OK;
}

int ext4pcf_to_map4(ext4pcf_ctx* ctx, const double* upsilon, const double* radial_bins, int n_bins,
                    int n_max, int n_phi, const double* ap_radii, int n_ap, const double* xi_acc, double* m4,
                    double* map4_eb, double* map4_disc) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  ctx->err.clear();
  if (!upsilon || !radial_bins || !ap_radii || !m4 || !map4_eb)
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "null pointer");
  if (n_bins < 1 || n_bins > 32 || n_max < 0 || n_max > 40 || n_phi < 1 || n_phi > 1024 || n_ap < 1 || n_ap > 64)
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "sizes out of range");
  for (int b = 0; b < n_bins; ++b)
    if (!(radial_bins[b + 1] > radial_bins[b]) || !(radial_bins[0] > 0))
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "radial_bins must increase from > 0");
  if (!is_device_ptr(upsilon)) return fail(ctx, EXT4PCF_E_INVALID_ARG, "upsilon must be a device pointer");
  if (real_space_smem(n_max, n_phi) > 227 * 1024) return fail(ctx, EXT4PCF_E_UNSUPPORTED, "n_max * n_phi too large");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = ctx->stream;
  const int ntri = n_bins * n_bins * n_bins;
  const size_t nph2 = (size_t)n_phi * n_phi;
  int chunk = (int)std::max<size_t>(1, (size_t)(256u << 20) / (nph2 * 8 * 16));
  if (chunk > ntri) chunk = ntri;
  ENSURE(ctx->t_norm, (size_t)chunk * nph2 * 8);
  ENSURE(ctx->t_gam, (size_t)chunk * nph2 * 8 * 16);
  ENSURE(ctx->t_E, (size_t)(2 * n_max + 1) * n_phi * 16);
  const int nsplit = map4_nsplit(chunk, ntri, n_ap);
  ENSURE(ctx->t_part, (size_t)ntri * nsplit * n_ap * 8 * 16);
  // small buffer: xi_acc [nb*6], tb [nb], area [nb], ap [n_ap], m4 [n_ap*16], eb [n_ap*16], disc [n_ap*16]
  const size_t small = (size_t)n_bins * 8 + n_ap * 49;
  ENSURE(ctx->t_small, small * 8);
  std::vector<double> hs(small, 0.0);
  double* h_tb = hs.data() + 6 * n_bins;
  double* h_area = h_tb + n_bins;
  double* h_ap = h_area + n_bins;
  for (int b = 0; b < n_bins; ++b) {
    const double lo = radial_bins[b], hi = radial_bins[b + 1];
    h_tb[b] = (2.0 / 3.0) * (hi * hi * hi - lo * lo * lo) / (hi * hi - lo * lo);
    h_area[b] = 0.5 * (hi * hi - lo * lo);
  }
  for (int k = 0; k < n_ap; ++k) h_ap[k] = ap_radii[k];
  double* d_small = (double*)ctx->t_small.p;
  CK(cudaMemcpyAsync(d_small, hs.data(), small * 8, cudaMemcpyHostToDevice, s));
  if (xi_acc)
    CK(cudaMemcpyAsync(d_small, xi_acc, (size_t)n_bins * 6 * 8,
                       is_device_ptr(xi_acc) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CK(map4_partials(upsilon, radial_bins, n_bins, n_max, n_phi, ap_radii, n_ap, (double*)ctx->t_E.p,
                   (double*)ctx->t_norm.p, (double*)ctx->t_gam.p, chunk, nsplit, (double*)ctx->t_part.p, s));
  double* d_m4 = d_small + 8 * n_bins + n_ap;
  double* d_eb = d_m4 + 16 * n_ap;
  double* d_disc = d_eb + 16 * n_ap;
  CK(map4_finish_launch((const double*)ctx->t_part.p, ntri * nsplit, n_ap, xi_acc ? d_small : nullptr, d_small + 6 * n_bins,
                        d_small + 7 * n_bins, n_bins, d_small + 8 * n_bins, d_m4, d_eb, d_disc, s));
  std::vector<double> res((size_t)48 * n_ap);
  CK(cudaMemcpyAsync(res.data(), d_m4, res.size() * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < 16 * n_ap; ++k) {
    m4[k] += res[k];
    map4_eb[k] += res[16 * n_ap + k];
    if (map4_disc && xi_acc) map4_disc[k] += res[32 * n_ap + k];
  }
  return EXT4PCF_OK;
}

int ext4pcf_measure3(ext4pcf_ctx* ctx, const double* positions, const double* shears, const double* weights,
                     int64_t n_gal, const double* radial_bins, int n_bins, int n_max, double* upsilon3) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  ctx->err.clear();
  if (n_gal < 0 || n_gal > (int64_t)2000000000) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_gal out of range");
  if (n_bins < 1 || n_bins > 32) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_bins must be in 1..32");
  if (n_max < 0 || n_max > 40) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_max must be in 0..40");
  if (!radial_bins || !upsilon3) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null radial_bins or upsilon3");
  if (n_gal > 0 && (!positions || !shears || !weights)) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null input");
  if (!(radial_bins[0] > 0.0) || !std::isfinite(radial_bins[n_bins]))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "radial_bins[0] must be > 0 and finite");
  for (int b = 0; b < n_bins; ++b)
    if (!(radial_bins[b + 1] > radial_bins[b])) return fail(ctx, EXT4PCF_E_INVALID_ARG, "radial_bins must increase");
  if (!is_device_ptr(upsilon3) ||
      (n_gal > 0 && (!is_device_ptr(positions) || !is_device_ptr(shears) || !is_device_ptr(weights))))
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "ext4pcf_measure3 takes device pointers");
  if (!contract3_supported(n_max)) return fail(ctx, EXT4PCF_E_UNSUPPORTED, "order-3 tables outside the record");
  CK(cudaSetDevice(ctx->cfg.device));
  if (n_gal == 0) return EXT4PCF_OK;
  cudaStream_t s = ctx->stream;
  const int nk = (int)n_gal;
  const size_t n = (size_t)n_gal;
  const Layout L = Layout::make(n_max, n_bins);
  Bins bins;
  bins.nb = n_bins;
  for (int b = 0; b <= n_bins; ++b) {
    bins.e2[b] = radial_bins[b] * radial_bins[b];
    bins.e2f[b] = (float)bins.e2[b];
  }
  bins.rmax = radial_bins[n_bins];
  // ---- grid (FP64 sorted catalogue)
  ENSURE(ctx->counter, 16);
  CK(cudaMemsetAsync(ctx->counter.p, 0, 8, s));
  ENSURE(ctx->bbox, (4 + 4 * 512) * 8);
  ENSURE(ctx->geom, sizeof(GridGeom));
  CK(grid_bbox(positions, nk, (double*)ctx->bbox.p, s));
  const int ntiles = (nk + 2047) / 2048;
  ENSURE(ctx->keys, n * 4); ENSURE(ctx->keys_alt, n * 4);
  ENSURE(ctx->perm, n * 4); ENSURE(ctx->perm_alt, n * 4);
  ENSURE(ctx->cell_start, grid_cells_cap(nk) * 4);
  ENSURE(ctx->hist, ((size_t)256 * ntiles * 2 + 4096) * 4);
  ENSURE(ctx->px, n * 8); ENSURE(ctx->py, n * 8);
  ENSURE(ctx->xr, n * 8); ENSURE(ctx->xi, n * 8); ENSURE(ctx->w, n * 8);
  // the gather runs in FP64 for EXT4PCF_FP64 and in FP32 (cell-anchored positions) otherwise
  const bool f64 = ctx->cfg.precision == EXT4PCF_FP64;
  if (!f64) { ENSURE(ctx->p4, n * 16); ENSURE(ctx->s4, n * 16); }
  GridBuffers gb;
  gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
  gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
  gb.cell_start = (int*)ctx->cell_start.p; gb.cell_cap = ctx->cell_start.bytes / 4;
  gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
  gb.px = (double*)ctx->px.p; gb.py = (double*)ctx->py.p;
  gb.xr = (double*)ctx->xr.p; gb.xi = (double*)ctx->xi.p; gb.w = (double*)ctx->w.p;
  gb.p4 = f64 ? nullptr : (float4*)ctx->p4.p; gb.s4 = f64 ? nullptr : (float4*)ctx->s4.p;
  gb.bbox = (double*)ctx->bbox.p;
  SortedCat cat;
  CK(grid_sort_device(positions, shears, weights, nk, 0, (const double*)ctx->bbox.p, bins.rmax,
                      (GridGeom*)ctx->geom.p, !f64, gb, cat, (int*)ctx->status.p, s));
  // ---- every galaxy a centre; waves of FP64 records, contracted with the order-3 tables
  ENSURE(ctx->centres, n * 4);
  iota<<<(nk + 255) / 256, 256, 0, s>>>((int*)ctx->centres.p, nk, 0);
  ++g_launches;
  CK(cudaGetLastError());
  const int T = std::min(ctx->cfg.wave_centres > 0 ? ctx->cfg.wave_centres : 4096, nk);
  const size_t cb = f64 ? sizeof(double2) : sizeof(float2);
  ENSURE(ctx->rec, (size_t)T * L.rec * cb);
  ENSURE(ctx->xw, (size_t)T * 2 * cb);
  ENSURE(ctx->corr, contract3_scratch_bytes(L, T));  // partial sums of the centre slices
  for (int w0 = 0; w0 < nk; w0 += T) {
    const int Tw = std::min(T, nk - w0);
    WavePlan P;
    P.nseg = 1;
    P.total = Tw;
    P.seg[0] = WaveSeg{(const int*)ctx->centres.p, nullptr, (const GridGeom*)ctx->geom.p, (const int*)ctx->cell_start.p,
                       w0, Tw, 0, 0, 0};
    if (f64) {
      GK(gather_wave<double>(cat, cat, bins, L, P, false, (double2*)ctx->rec.p, (double2*)ctx->xw.p,
                             (unsigned long long*)ctx->counter.p, ctx->sm_count, s));
      CK(contract3_wave(L, (const double2*)ctx->rec.p, (const double2*)ctx->xw.p, Tw, upsilon3,
                        (double2*)ctx->corr.p, s));
    } else {
      GK(gather_wave<float>(cat, cat, bins, L, P, false, (float2*)ctx->rec.p, (float2*)ctx->xw.p,
                            (unsigned long long*)ctx->counter.p, ctx->sm_count, s));
      CK(contract3_wave(L, (const float2*)ctx->rec.p, (const float2*)ctx->xw.p, Tw, upsilon3,
                        (double2*)ctx->corr.p, s));
    }
  }
  CK(cudaGetLastError());
  return EXT4PCF_OK;
}

int ext4pcf_map_direct(ext4pcf_ctx* ctx, const double* positions, const double* shears, const double* weights,
                       int64_t n_gal, const double* thetas, int n_theta, const double* centres,
                       const int64_t* centre_offsets, double* ap_records, double* moments) {
  if (!ctx) return EXT4PCF_E_INVALID_ARG;
  ctx->err.clear();
  if (!thetas || !centre_offsets || !moments || n_theta < 1 || n_theta > 4096)
    return fail(ctx, EXT4PCF_E_INVALID_ARG, "thetas, centre_offsets and moments are required (1 <= n_theta <= 4096)");
  if (n_gal < 0 || n_gal > 2147483647LL) return fail(ctx, EXT4PCF_E_INVALID_ARG, "n_gal out of range");
  if (n_gal > 0 && (!positions || !shears || !weights)) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null catalogue");
  double tmin = 0, tmax = 0;
  for (int t = 0; t < n_theta; ++t) {
    if (!(thetas[t] > 0) || !std::isfinite(thetas[t]))
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "aperture radii must be finite and > 0");
    tmin = t ? std::fmin(tmin, thetas[t]) : thetas[t];
    tmax = t ? std::fmax(tmax, thetas[t]) : thetas[t];
  }
  if (centre_offsets[0] != 0) return fail(ctx, EXT4PCF_E_INVALID_ARG, "centre_offsets[0] must be 0");
  for (int t = 0; t < n_theta; ++t)
    if (centre_offsets[t + 1] < centre_offsets[t] || centre_offsets[t + 1] - centre_offsets[t] > 2147483647LL)
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "centre_offsets must be non-decreasing");
  const int64_t n_cen = centre_offsets[n_theta];
  if (n_cen > 0 && !centres) return fail(ctx, EXT4PCF_E_INVALID_ARG, "null centres");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = ctx->stream;
  const size_t n = (size_t)n_gal;
  // ---- stage host inputs / outputs
  const double* d_pos = positions;
  const double* d_sh = shears;
  const double* d_w = weights;
  const double* d_cen = centres;
  if (n > 0 && !is_device_ptr(positions)) {
    ENSURE(ctx->in_pos, n * 16);
    CK(cudaMemcpyAsync(ctx->in_pos.p, positions, n * 16, cudaMemcpyHostToDevice, s));
    d_pos = (const double*)ctx->in_pos.p;
  }
  if (n > 0 && !is_device_ptr(shears)) {
    ENSURE(ctx->in_shear, n * 16);
    CK(cudaMemcpyAsync(ctx->in_shear.p, shears, n * 16, cudaMemcpyHostToDevice, s));
    d_sh = (const double*)ctx->in_shear.p;
  }
  if (n > 0 && !is_device_ptr(weights)) {
    ENSURE(ctx->in_w, n * 8);
    CK(cudaMemcpyAsync(ctx->in_w.p, weights, n * 8, cudaMemcpyHostToDevice, s));
    d_w = (const double*)ctx->in_w.p;
  }
  if (n_cen > 0 && !is_device_ptr(centres)) {
    ENSURE(ctx->ap_cen, (size_t)n_cen * 16);
    CK(cudaMemcpyAsync(ctx->ap_cen.p, centres, (size_t)n_cen * 16, cudaMemcpyHostToDevice, s));
    d_cen = (const double*)ctx->ap_cen.p;
  }
  const bool host_rec = ap_records && !is_device_ptr(ap_records);
  double* d_rec = ap_records;
  if (!ap_records || host_rec) {
    ENSURE(ctx->io_rec, (size_t)n_cen * 64);
    d_rec = (double*)ctx->io_rec.p;
  }
  const bool host_mom = !is_device_ptr(moments);
  double* d_mom = moments;
  if (host_mom) {
    ENSURE(ctx->io_mom, (size_t)n_theta * 64);
    CK(cudaMemcpyAsync(ctx->io_mom.p, moments, (size_t)n_theta * 64, cudaMemcpyHostToDevice, s));
    d_mom = (double*)ctx->io_mom.p;
  }
  // ---- grid: power-of-two cells (exact float corner arithmetic), about eight per cut
  // radius of the smallest aperture, at most ~4096 per axis and per largest cut diameter
  SortedCat cat;
  cat.n = 0;
  double cell = 1.0;
  if (n > 0) {
    const int nk = (int)n;
    ENSURE(ctx->bbox, (4 + 4 * 512) * 8);
    CK(grid_bbox(d_pos, nk, (double*)ctx->bbox.p, s));
    double bb[4];
    CK(cudaMemcpyAsync(bb, ctx->bbox.p, 32, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!std::isfinite(bb[0]) || !std::isfinite(bb[1]) || !std::isfinite(bb[2]) || !std::isfinite(bb[3]))
      return fail(ctx, EXT4PCF_E_INVALID_ARG, "non-finite positions");
    const double extent = std::fmax(bb[2] - bb[0], bb[3] - bb[1]);
    const double target = std::fmax(0.5 * tmin, std::fmax(extent / 2048.0, 4.0 * tmax / 2048.0));
    int ex;
    std::frexp(target, &ex);
    cell = std::ldexp(1.0, ex - 1);  // largest power of two <= target
    const int ncx = (int)std::floor((bb[2] - bb[0]) / cell) + 1;
    const int ncy = (int)std::floor((bb[3] - bb[1]) / cell) + 1;
    const size_t ncells = (size_t)ncx * ncy;
    const int ntiles = (nk + 2047) / 2048;
    ENSURE(ctx->keys, n * 4); ENSURE(ctx->keys_alt, n * 4);
    ENSURE(ctx->perm, n * 4); ENSURE(ctx->perm_alt, n * 4);
    ENSURE(ctx->cell_start, (ncells + 1) * 4);
    ENSURE(ctx->hist, ((size_t)256 * ntiles * 2 + 4096) * 4);
    ENSURE(ctx->px, n * 8); ENSURE(ctx->py, n * 8);
    ENSURE(ctx->xr, n * 8); ENSURE(ctx->xi, n * 8); ENSURE(ctx->w, n * 8);
    ENSURE(ctx->p4, n * 16); ENSURE(ctx->s4, n * 16);
    GridBuffers gb;
    gb.keys = (int*)ctx->keys.p; gb.keys_alt = (int*)ctx->keys_alt.p;
    gb.perm = (int*)ctx->perm.p; gb.perm_alt = (int*)ctx->perm_alt.p;
    gb.cell_start = (int*)ctx->cell_start.p; gb.cell_cap = ncells + 1;
    gb.hist = (unsigned*)ctx->hist.p; gb.hist_cap = ctx->hist.bytes / 4;
    gb.px = (double*)ctx->px.p; gb.py = (double*)ctx->py.p;
    gb.xr = (double*)ctx->xr.p; gb.xi = (double*)ctx->xi.p; gb.w = (double*)ctx->w.p;
    gb.p4 = (float4*)ctx->p4.p; gb.s4 = (float4*)ctx->s4.p; gb.bbox = (double*)ctx->bbox.p;
    CK(grid_sort(d_pos, d_sh, d_w, nk, bb[0], bb[1], cell, ncx, ncy, true, gb, cat, s));
  }
  // ---- apertures, one radius at a time
  size_t sums_need = 16;
  std::vector<int> splits(n_theta);
  for (int t = 0; t < n_theta; ++t) {
    const int na = (int)(centre_offsets[t + 1] - centre_offsets[t]);
    splits[t] = map_direct_splits(na, ctx->sm_count, thetas[t], cell);
    sums_need = std::max(sums_need, map_direct_scratch(na, splits[t]));
  }
  ENSURE(ctx->ap_sums, sums_need);
  for (int t = 0; t < n_theta; ++t) {
    const int64_t c0 = centre_offsets[t];
    const int na = (int)(centre_offsets[t + 1] - c0);
    CK(map_direct_radius(cat, d_cen + 2 * c0, na, thetas[t], splits[t], ctx->ap_sums.p, d_rec + 8 * c0,
                         d_mom + 8 * t, s));
  }
  if (host_rec && n_cen > 0)
    CK(cudaMemcpyAsync(ap_records, d_rec, (size_t)n_cen * 64, cudaMemcpyDeviceToHost, s));
  if (host_mom) CK(cudaMemcpyAsync(moments, d_mom, (size_t)n_theta * 64, cudaMemcpyDeviceToHost, s));
  if (host_rec || host_mom) CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return EXT4PCF_OK;
}

}  // extern "C"
