// ig_api.cu -- the C ABI (include/iskra_gb300.h): argument checks, device memory ownership and
// the order of kernel launches. No arithmetic of the method happens here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>

#include "ig_internal.cuh"

namespace ig {

void set_error(ig_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
}

namespace {
struct ProfState {
  std::mutex mu;
  bool on = false;
  struct Rec {
    const char* name;
    cudaEvent_t e0, e1;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<int64_t, double>> acc;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& r : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
        auto& a = acc[r.name];
        a.first += 1;
        a.second += ms;
      }
      cudaGetLastError();
      pool.push_back(r.e0);
      pool.push_back(r.e1);
    }
    pending.clear();
  }
};
ProfState& prof_state() {
  static ProfState* s = new ProfState();
  return *s;
}
}  // namespace

bool prof_on() { return prof_state().on; }

ProfScope::ProfScope(const char* n, cudaStream_t s) : name(n), st(s) {
  ProfState& P = prof_state();
  if (!P.on) return;
  std::lock_guard<std::mutex> lk(P.mu);
  cudaEvent_t e0 = P.get(), e1 = P.get();
  if (!e0 || !e1) return;
  cudaEventRecord(e0, st);
  P.pending.push_back({name, e0, e1});
  slot = (int)P.pending.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  ProfState& P = prof_state();
  std::lock_guard<std::mutex> lk(P.mu);
  cudaEventRecord(P.pending[slot].e1, st);
  if (P.pending.size() > 4096) P.drain();
}

}  // namespace ig

using namespace ig;

namespace {

ig_status from_cuda(ig_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return IG_OK;
  set_error(ctx, std::string(where) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return IG_ERR_OOM;
  }
  return IG_ERR_CUDA;
}

#define IG_CK(ctx, call, where)                                        \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return from_cuda((ctx), e_, (where));       \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ig_status bad_arg(ig_ctx* ctx, const char* msg) {
  set_error(ctx, msg);
  return IG_ERR_INVALID_ARG;
}

template <typename T>
cudaError_t mesh_alloc(ig_mesh* mesh, T** out, size_t count) {
  void* p = nullptr;
  const size_t bytes = sizeof(T) * (count > 0 ? count : 1);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return e;
  mesh->allocs.push_back(p);
  mesh->bytes += (int64_t)bytes;
  *out = static_cast<T*>(p);
  return cudaSuccess;
}

void mesh_release(ig_mesh* mesh) {
  group_destroy(mesh->group);
  for (void* p : mesh->allocs) cudaFree(p);
  mesh->allocs.clear();
}

ig_status err_bits_to_status(int bits) {
  if (bits & (kErrIndex | kErrBounds)) return IG_ERR_INDEX_OUT_OF_RANGE;
  if (bits & kErrRepeated) return IG_ERR_DEGENERATE_FACE;
  if (bits & kErrNonfinite) return IG_ERR_NONFINITE;
  if (bits & kErrDegenerate) return IG_ERR_DEGENERATE_FACE;
  if (bits & (kErrUnused | kErrValence)) return IG_ERR_INVALID_ARG;
  return IG_OK;
}

const char* err_bits_message(int bits) {
  if (bits & kErrBounds) return "an index read from device data was out of range (bounds-checked build)";
  if (bits & kErrIndex) return "a face index is outside [0, n)";
  if (bits & kErrRepeated) return "a face repeats a vertex";
  if (bits & kErrNonfinite) return "a vertex position is not finite";
  if (bits & kErrDegenerate) return "a face has zero area";
  if (bits & kErrUnused) return "a vertex is used by no face";
  if (bits & kErrValence) return "a vertex has more than 65535 neighbours";
  return "";
}

// Device temporaries released when the owner goes out of scope.
struct TmpAllocs {
  std::vector<void*> v;
  ~TmpAllocs() {
    for (void* p : v) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1));
    if (e == cudaSuccess) {
      v.push_back(p);
      *out = static_cast<T*>(p);
    }
    return e;
  }
};

ig_solve_opts resolve_opts(const ig_solve_opts* o) {
  ig_solve_opts d;
  ig_default_opts(&d);
  return o ? *o : d;
}

ig_status check_opts(ig_ctx* ctx, const ig_solve_opts& o) {
  if (!(o.rel_tol >= 0.0) || !std::isfinite(o.rel_tol)) return bad_arg(ctx, "rel_tol must be finite and >= 0");
  if (o.max_iter < 1 || o.max_iter > 100000000) return bad_arg(ctx, "max_iter must be in [1, 1e8]");
  if (o.launch != IG_LAUNCH_GRAPH && o.launch != IG_LAUNCH_HOST) return bad_arg(ctx, "unknown launch mode");
  if (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0)) return bad_arg(ctx, "inner_tol must be in (0, 1)");
  if (o.max_refine < 1) return bad_arg(ctx, "max_refine must be >= 1");
  return IG_OK;
}

// Synchronise, then report the solve state of the mesh into info and as a status.
ig_status collect_info(ig_mesh* mesh, int k, ig_solve_info* info) {
  ig_ctx* ctx = mesh->ctx;
  SolveScal s;
  int bits = 0;
  IG_CK(ctx, cudaMemcpyAsync(&s, mesh->md.s, sizeof(SolveScal), cudaMemcpyDeviceToHost, ctx->stream), "read state");
  IG_CK(ctx, cudaMemcpyAsync(&bits, mesh->md.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read state");
  IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "solve");
  ig_status st = (ig_status)s.status;
  if (bits) {
    st = err_bits_to_status(bits);
    set_error(ctx, err_bits_message(bits));
  } else if (st == IG_ERR_NOT_CONVERGED) {
    set_error(ctx, "conjugate gradients reached max_iter above rel_tol");
  } else if (st == IG_ERR_NONFINITE) {
    set_error(ctx, "non-finite value or breakdown in conjugate gradients");
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = st;
    info->k = k;
    info->iterations = s.iter;
    info->refinements = s.refine;
    for (int c = 0; c < kMaxK; ++c) {
      info->rel_residual[c] = c < k ? s.relres[c] : 0.0;
      info->true_rel_residual[c] = c < k ? s.trueres[c] : 0.0;
    }
  }
  return st;
}

}  // namespace

namespace ig {

// Allocate the FP32 copies used by mixed precision (once per mesh) and refresh the mesh's own
// descriptor on the device.
cudaError_t mesh_ensure_mixed(ig_mesh* mesh, cudaStream_t st) {
  MeshDev& md = mesh->md;
  if (md.A32) return cudaSuccess;
  const size_t nv = (size_t)mesh->n * kMaxK;
  cudaError_t e;
  if ((e = mesh_alloc(mesh, &md.A32, (size_t)md.nnz_sell)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(md.A32, 0, sizeof(float) * (size_t)md.nnz_sell, st)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.Dinv32, (size_t)mesh->n)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.x32, nv)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.r32, nv)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.p32, nv)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.q32, nv)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(md.p32, 0, sizeof(float) * nv, st)) != cudaSuccess) return e;
  if (md.sell_ptr) {
    // 16-bit column offsets, kept when every slice's columns fit (one-time check on the host)
    short* c16 = nullptr;
    int* nfar = nullptr;
    if ((e = mesh_alloc(mesh, &c16, (size_t)md.nnz_sell)) != cudaSuccess) return e;
    if ((e = mesh_alloc(mesh, &nfar, 1)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(nfar, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = launch_sell_c16(md.sell_ptr, md.sell_col, mesh->n, c16, nfar, st)) != cudaSuccess) return e;
    int far = 1;
    if ((e = cudaMemcpyAsync(&far, nfar, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    md.sell_c16 = far == 0 ? c16 : nullptr;
  }
  mesh->group.host_mds[0] = md;
  return group_upload_mds(mesh->group, st);
}

// The buffers of FP32 face geometry (once per mesh): split positions, split U and Lambda and the
// per-vertex weights of the gradient; the per-face weights and gradients reuse facew and gface.
cudaError_t mesh_ensure_geom32(ig_mesh* mesh, cudaStream_t st) {
  cudaError_t e = mesh_ensure_mixed(mesh, st);
  if (e != cudaSuccess) return e;
  MeshDev& md = mesh->md;
  if (md.vsplit) return cudaSuccess;
  const size_t n = (size_t)mesh->n;
  if ((e = mesh_alloc(mesh, &md.vsplit, 8 * n)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.usplit, 8 * n)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.lsplit, 8 * n)) != cudaSuccess) return e;
  if ((e = mesh_alloc(mesh, &md.wv, n)) != cudaSuccess) return e;
  mesh->group.host_mds[0] = md;
  return group_upload_mds(mesh->group, st);
}

// Record the geometry mode of the next assembly in the mesh's descriptor (host and device copies).
cudaError_t mesh_set_geom32(ig_mesh* mesh, int geom32, cudaStream_t st) {
  if (mesh->md.geom32 == geom32) return cudaSuccess;
  mesh->md.geom32 = geom32;
  mesh->group.host_mds[0] = mesh->md;
  return group_upload_mds(mesh->group, st);
}

}  // namespace ig

// =============================================================================================
extern "C" {

const char* ig_status_str(ig_status s) {
  switch (s) {
    case IG_OK: return "ok";
    case IG_ERR_INVALID_ARG: return "invalid argument";
    case IG_ERR_INDEX_OUT_OF_RANGE: return "face index out of range";
    case IG_ERR_DEGENERATE_FACE: return "degenerate face";
    case IG_ERR_NOT_CONVERGED: return "solver did not converge";
    case IG_ERR_NONFINITE: return "non-finite value";
    case IG_ERR_OOM: return "out of device memory";
    case IG_ERR_CUDA: return "CUDA error";
    case IG_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

void ig_default_opts(ig_solve_opts* o) {
  if (!o) return;
  o->rel_tol = 1e-10;
  o->max_iter = 20000;
  o->launch = IG_LAUNCH_GRAPH;
  o->inner_tol = 1e-5;
  o->max_refine = 30;
}

ig_status ig_create(ig_ctx** out, int device, void* cuda_stream) {
  IG_NVTX("ig_create");
  if (!out) return IG_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return IG_ERR_CUDA;
  }
  ig_ctx* ctx = new (std::nothrow) ig_ctx();
  if (!ctx) return IG_ERR_OOM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return IG_ERR_CUDA;
  }
  ctx->solver_slots = ctx->num_sms * solver_blocks_per_sm();
  ctx->solver_slots32 = ctx->num_sms * solver_blocks_per_sm_mixed();
  cudaGetLastError();
  *out = ctx;
  return IG_OK;
}

ig_status ig_set_stream(ig_ctx* ctx, void* cuda_stream) {
  if (!ctx) return IG_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return IG_OK;
}

ig_status ig_destroy(ig_ctx* ctx) {
  IG_NVTX("ig_destroy");
  if (!ctx) return IG_ERR_INVALID_ARG;
  if (ctx->live_meshes != 0) return bad_arg(ctx, "meshes still alive on this context");
  delete ctx;
  return IG_OK;
}

const char* ig_last_error(ig_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

ig_status ig_mesh_upload(ig_ctx* ctx, const int32_t* F_dev, int64_t m, int64_t n, ig_mesh** out) {
  IG_NVTX("ig_mesh_upload");
  if (!ctx || !out) return IG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!F_dev) return bad_arg(ctx, "F is NULL");
  if (n < 3 || m < 1) return bad_arg(ctx, "need n >= 3 and m >= 1");
  if (n > (1ll << 30) || m > (1ll << 29)) return bad_arg(ctx, "mesh too large for 32-bit offsets");
  DeviceGuard guard(ctx->device);
  cudaStream_t st = ctx->stream;
  std::unique_ptr<ig_mesh> mesh(new (std::nothrow) ig_mesh());
  if (!mesh) return IG_ERR_OOM;
  ig_mesh* M = mesh.get();
  M->ctx = ctx;
  M->n = n;
  M->m = m;
  const int ni = (int)n, mi = (int)m;

  TmpAllocs tmp;  // temporaries, freed before returning

  int *F = nullptr, *incptr = nullptr, *rowptr = nullptr, *diagpos = nullptr, *err = nullptr, *col = nullptr;
  int2* inc = nullptr;
  int *deg = nullptr, *fill = nullptr, *inc_fc = nullptr, *nbr = nullptr, *rowlen = nullptr, *scratch = nullptr,
      *totals = nullptr;
  ig_status rs = IG_OK;
  auto fail = [&](cudaError_t e, const char* where) {
    rs = from_cuda(ctx, e, where);
    mesh_release(M);
    return rs;
  };
#define UP_CK(call, where)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return fail(e_, where);  \
  } while (0)

  const size_t scan_ints = scan_scratch_ints(std::max(ni, 3 * mi) + 1);
  UP_CK(mesh_alloc(M, &F, 3 * (size_t)m), "alloc F");
  UP_CK(mesh_alloc(M, &incptr, (size_t)n + 1), "alloc incptr");
  UP_CK(mesh_alloc(M, &rowptr, (size_t)n + 1), "alloc rowptr");
  UP_CK(mesh_alloc(M, &diagpos, (size_t)n), "alloc diagpos");
  UP_CK(mesh_alloc(M, &inc, 3 * (size_t)m), "alloc incidence");
  UP_CK(mesh_alloc(M, &err, 1), "alloc err");
  UP_CK(tmp.get(&deg, (size_t)n), "alloc tmp");
  UP_CK(tmp.get(&fill, (size_t)n), "alloc tmp");
  UP_CK(tmp.get(&inc_fc, 3 * (size_t)m), "alloc tmp");
  UP_CK(tmp.get(&nbr, 6 * (size_t)m + (size_t)n), "alloc tmp");
  UP_CK(tmp.get(&rowlen, (size_t)n), "alloc tmp");
  UP_CK(tmp.get(&scratch, scan_ints), "alloc tmp");
  UP_CK(tmp.get(&totals, 2), "alloc tmp");

  UP_CK(cudaMemcpyAsync(F, F_dev, sizeof(int) * 3 * (size_t)m, cudaMemcpyDeviceToDevice, st), "copy F");
  UP_CK(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)n, st), "memset");
  UP_CK(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)n, st), "memset");
  UP_CK(cudaMemsetAsync(err, 0, sizeof(int), st), "memset");
  UP_CK(launch_pattern_count(F, mi, ni, deg, err, st), "pattern count");
  UP_CK(exclusive_scan_int(deg, incptr, ni, totals, scratch, scan_ints, st), "scan");
  int host_err = 0;
  UP_CK(cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, st), "read err");
  UP_CK(cudaStreamSynchronize(st), "pattern count");
  if (host_err) {
    set_error(ctx, err_bits_message(host_err));
    mesh_release(M);
    return err_bits_to_status(host_err);
  }
  UP_CK(launch_pattern_fill(F, mi, incptr, fill, inc_fc, st), "pattern fill");
  UP_CK(launch_pattern_rows(F, ni, incptr, inc_fc, nbr, rowlen, err, st), "pattern rows");
  UP_CK(exclusive_scan_int(rowlen, rowptr, ni, totals + 1, scratch, scan_ints, st), "scan");
  int host_tot[2] = {0, 0};
  UP_CK(cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, st), "read err");
  UP_CK(cudaMemcpyAsync(host_tot, totals, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "read totals");
  UP_CK(cudaStreamSynchronize(st), "pattern rows");
  if (host_err) {
    set_error(ctx, err_bits_message(host_err));
    mesh_release(M);
    return err_bits_to_status(host_err);
  }
  const int nnz = host_tot[1];
  M->nnz = nnz;
  UP_CK(mesh_alloc(M, &col, (size_t)nnz), "alloc col");
  UP_CK(launch_pattern_cols(F, ni, incptr, inc_fc, nbr, rowptr, col, diagpos, inc, err, st), "pattern cols");

  // sliced-ELL copy of the pattern for the solver's SpMV (slices of 32 rows)
  const int nsl = (ni + 31) / 32;
  int *width32 = nullptr, *sell_ptr = nullptr, *sell_col = nullptr;
  UP_CK(tmp.get(&width32, (size_t)nsl), "alloc tmp");
  UP_CK(mesh_alloc(M, &sell_ptr, (size_t)nsl + 1), "alloc sell");
  UP_CK(launch_sell_width(rowptr, ni, width32, st), "sell width");
  UP_CK(exclusive_scan_int(width32, sell_ptr, nsl, totals, scratch, scan_ints, st), "scan");
  int nnz_sell = 0;
  std::vector<int> widths((size_t)nsl);
  UP_CK(cudaMemcpyAsync(&nnz_sell, totals, sizeof(int), cudaMemcpyDeviceToHost, st), "read totals");
  UP_CK(cudaMemcpyAsync(widths.data(), width32, sizeof(int) * (size_t)nsl, cudaMemcpyDeviceToHost, st),
        "read widths");
  UP_CK(cudaStreamSynchronize(st), "sell width");
  // When padding every slice to the widest one costs at most 1/64 more entries (a grid: only the
  // slices of its first and last row of vertices are narrower), all slices get that width and
  // the SpMV computes a slice's offset instead of loading it.
  int sell_w = 0;
  {
    long wmax = 0;
    for (int w : widths) wmax = w > wmax ? w : wmax;
    const long padded = wmax * (long)nsl;
    if (nsl > 0 && padded <= (long)nnz_sell + (long)nnz_sell / 64 && padded < (long)INT32_MAX) {
      std::vector<int> ptr((size_t)nsl + 1);
      for (long s2 = 0; s2 <= nsl; ++s2) ptr[(size_t)s2] = (int)(s2 * wmax);
      UP_CK(cudaMemcpyAsync(sell_ptr, ptr.data(), sizeof(int) * ((size_t)nsl + 1), cudaMemcpyHostToDevice, st),
            "sell ptr");
      UP_CK(cudaStreamSynchronize(st), "sell ptr");
      nnz_sell = (int)padded;
      sell_w = (int)(wmax / 32);
    }
  }
  UP_CK(mesh_alloc(M, &sell_col, (size_t)nnz_sell), "alloc sell");
  UP_CK(launch_sell_fill(rowptr, col, ni, sell_ptr, sell_col, st), "sell fill");

  // operator and solver workspace
  MeshDev& md = M->md;
  std::memset(&md, 0, sizeof(md));
  md.n = ni;
  md.m = mi;
  md.nnz = nnz;
  // Solver tiles (whole warps, at least kBlock rows): the choice depends on n and the device only,
  // never on a batch.
  // Mixed precision: 256..max_rows rows; a mesh that fills the GPU gets a tile count that is a
  // whole multiple of the resident CTA slots S of the solver kernels, so every launch ends in full
  // waves. The SpMV and the p-update take one pass (kTileRows rows) per tile: a big mesh's tiles
  // are dealt cyclically, so CTAs at work at the same time cover neighbouring rows and share the
  // gathered p lines in L2. The update gathers nothing; on a big mesh it takes one wave of large
  // tiles (up to kMaxTileRows32 rows, in passes of kTileRows), which costs far fewer barriers and
  // partial sums (one-wave tiles measured 139.9 -> 113.7 us per update launch on the 4096 x 2048
  // grid, and 139.2 -> 159.5 us per SpMV launch, hence the two tilings).
  auto choose_tiles = [ni](long S, long max_rows, int& tile_rows, int& ntiles) {
    if (S < 1) S = 1;
    long waves = ((long)ni + S * max_rows - 1) / (S * max_rows);
    if (waves < 1) waves = 1;
    long rows = ((long)ni + S * waves - 1) / (S * waves);
    if (rows < kBlock) rows = kBlock;
    if (rows > max_rows) rows = max_rows;
    rows = (rows + 31) / 32 * 32;
    tile_rows = (int)rows;
    ntiles = (int)(((long)ni + rows - 1) / rows);
  };
  // FP64: a CTA takes a tile in passes of kBlock rows (one row per thread), and its warps meet at
  // the tile's reduction, so a last pass that is only partly filled leaves most warps waiting.
  // For w waves of tiles (rows = n / (S w), at most kTileRows64) a CTA makes w * ceil(rows /
  // kBlock) passes; the tiling takes the w with the fewest passes, counting each tile's
  // reduction as a quarter pass. 1,048,576 rows on 608 slots: one wave of 1728-row tiles
  // (7 passes) where two waves of 864-row tiles took 2 x 4.
  auto choose_tiles64 = [ni](long S, int& tile_rows, int& ntiles) {
    if (S < 1) S = 1;
    long w0 = ((long)ni + S * kTileRows64 - 1) / (S * kTileRows64);
    if (w0 < 1) w0 = 1;
    long best_rows = kBlock, best_cost = -1;
    for (long w = w0; w < w0 + 64; ++w) {
      long r = ((long)ni + S * w - 1) / (S * w);
      r = (r + 31) / 32 * 32;
      if (r < kBlock) r = kBlock;
      const long cost = 4 * w * ((r + kBlock - 1) / kBlock) + w;  // in quarter passes
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        best_rows = r;
      }
      if (r == kBlock) break;  // more waves only add passes
    }
    tile_rows = (int)best_rows;
    ntiles = (int)(((long)ni + best_rows - 1) / best_rows);
  };
  choose_tiles64(ctx->solver_slots, md.tile_rows, md.ntiles);
  choose_tiles(ctx->solver_slots32, kTileRows, md.tile_rows32, md.ntiles32);
  if (ni >= kBigRows) {
    choose_tiles(ctx->solver_slots32, kMaxTileRows32, md.tile_rows32u, md.ntiles32u);
  } else {
    md.tile_rows32u = md.tile_rows32;
    md.ntiles32u = md.ntiles32;
  }
  md.nnz_sell = nnz_sell;
  md.sell_w = sell_w;
  md.sell_ptr = sell_ptr;
  md.sell_col = sell_col;
  md.F = F;
  md.rowptr = rowptr;
  md.col = col;
  md.diagpos = diagpos;
  md.incptr = incptr;
  md.inc = inc;
  md.err = err;
  const size_t nv = (size_t)n * kMaxK;
  // partial sums: the loop kernels' tiles (twice over for the cluster loop of small meshes, which
  // keeps the SpMV's and the update's partials apart), and the VJP's per-face-tile sums of dl/dt
  const size_t npart = std::max(std::max((size_t)md.ntiles, (size_t)md.ntiles32) * 2 * kPartStride,
                                (size_t)(mi + 255) / 256) + 8;
  UP_CK(mesh_alloc(M, &md.facew, 4 * (size_t)m), "alloc");
  UP_CK(mesh_alloc(M, &md.A, (size_t)nnz_sell), "alloc");
  UP_CK(cudaMemsetAsync(md.A, 0, sizeof(double) * (size_t)nnz_sell, st), "memset");
  UP_CK(mesh_alloc(M, &md.M, (size_t)n), "alloc");
  UP_CK(mesh_alloc(M, &md.Dinv, (size_t)n), "alloc");
  UP_CK(mesh_alloc(M, &md.x, nv), "alloc");
  UP_CK(mesh_alloc(M, &md.r, nv), "alloc");
  UP_CK(mesh_alloc(M, &md.p, nv), "alloc");
  UP_CK(mesh_alloc(M, &md.q, nv), "alloc");
  UP_CK(mesh_alloc(M, &md.z, nv), "alloc");
  md.rhs = md.q;  // the FP64 q vector is unused in mixed precision, where it keeps the rhs
  UP_CK(mesh_alloc(M, &md.lam, nv), "alloc");
  UP_CK(mesh_alloc(M, &md.gface, 9 * (size_t)m), "alloc");
  UP_CK(mesh_alloc(M, &md.part, npart), "alloc");
  UP_CK(mesh_alloc(M, &md.s, 1), "alloc");
  UP_CK(cudaMemsetAsync(md.s, 0, sizeof(SolveScal), st), "memset");
  UP_CK(cudaMemsetAsync(md.p, 0, sizeof(double) * nv, st), "memset");
  UP_CK(cudaMemsetAsync(md.q, 0, sizeof(double) * nv, st), "memset");
  UP_CK(cudaMemsetAsync(md.z, 0, sizeof(double) * nv, st), "memset");
  UP_CK(group_init(M->group, &md, 1, ctx->solver_slots, ctx->solver_slots32, st), "group");
  UP_CK(cudaStreamSynchronize(st), "upload");
#undef UP_CK
  ctx->live_meshes += 1;
  *out = mesh.release();
  return IG_OK;
}

ig_status ig_mesh_free(ig_mesh* mesh) {
  IG_NVTX("ig_mesh_free");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  mesh_release(mesh);
  ctx->live_meshes -= 1;
  delete mesh;
  return IG_OK;
}

ig_status ig_mesh_info(ig_mesh* mesh, int64_t* n, int64_t* m, int64_t* nnz, int64_t* device_bytes) {
  if (!mesh) return IG_ERR_INVALID_ARG;
  if (n) *n = mesh->n;
  if (m) *m = mesh->m;
  if (nnz) *nnz = mesh->nnz;
  if (device_bytes) *device_bytes = mesh->bytes;
  return IG_OK;
}

ig_status ig_mesh_pattern(ig_mesh* mesh, int32_t* rowptr_dev, int32_t* col_dev) {
  IG_NVTX("ig_mesh_pattern");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  DeviceGuard guard(ctx->device);
  if (rowptr_dev)
    IG_CK(ctx, cudaMemcpyAsync(rowptr_dev, mesh->md.rowptr, sizeof(int) * (mesh->n + 1), cudaMemcpyDeviceToDevice,
                               ctx->stream), "copy rowptr");
  if (col_dev)
    IG_CK(ctx, cudaMemcpyAsync(col_dev, mesh->md.col, sizeof(int) * mesh->nnz, cudaMemcpyDeviceToDevice, ctx->stream),
          "copy col");
  return IG_OK;
}

ig_status ig_assemble(ig_mesh* mesh, const double* V_dev, double t, int precision) {
  IG_NVTX("ig_assemble");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev) return bad_arg(ctx, "V is NULL");
  if (!(t >= 0.0) || !std::isfinite(t)) return bad_arg(ctx, "t must be finite and >= 0");
  if (precision != IG_PRECISION_FP64 && precision != IG_PRECISION_MIXED && precision != IG_PRECISION_MIXED_GEOM32)
    return bad_arg(ctx, "unknown precision");
  DeviceGuard guard(ctx->device);
  if (precision == IG_PRECISION_MIXED) IG_CK(ctx, mesh_ensure_mixed(mesh, ctx->stream), "alloc");
  if (precision == IG_PRECISION_MIXED_GEOM32) IG_CK(ctx, mesh_ensure_geom32(mesh, ctx->stream), "alloc");
  IG_CK(ctx, mesh_set_geom32(mesh, precision == IG_PRECISION_MIXED_GEOM32 ? 1 : 0, ctx->stream), "upload");
  CallDev call{};
  call.V = V_dev;
  call.t = t;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, cudaMemsetAsync(mesh->md.err, 0, sizeof(int), ctx->stream), "memset");
  IG_CK(ctx, launch_assemble(mesh->group, precision, ctx->stream), "assemble");
  mesh->assembled = precision + 1;  // 1 FP64, 2 mixed, 3 mixed with FP32 geometry
  mesh->t = t;
  return IG_OK;
}

ig_status ig_mesh_set_cot_clamp(ig_mesh* mesh, int enable, double clamp_min) {
  IG_NVTX("ig_mesh_set_cot_clamp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (enable && !std::isfinite(clamp_min)) return bad_arg(ctx, "clamp_min must be finite");
  DeviceGuard guard(ctx->device);
  mesh->md.clamp_on = enable ? 1 : 0;
  mesh->md.clamp_min = enable ? clamp_min : 0.0;
  mesh->group.host_mds[0] = mesh->md;
  IG_CK(ctx, group_upload_mds(mesh->group, ctx->stream), "upload");
  mesh->assembled = 0;  // the operator must be assembled again with the new weights
  return IG_OK;
}

ig_status ig_check(ig_mesh* mesh) {
  IG_NVTX("ig_check");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  DeviceGuard guard(ctx->device);
  int bits = 0;
  IG_CK(ctx, cudaMemcpyAsync(&bits, mesh->md.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read err");
  IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "check");
  if (bits) set_error(ctx, err_bits_message(bits));
  return err_bits_to_status(bits);
}

ig_status ig_operator(ig_mesh* mesh, double* Aval_dev, double* M_dev) {
  IG_NVTX("ig_operator");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled) {
    set_error(ctx, "operator requested before assemble");
    return IG_ERR_STATE;
  }
  DeviceGuard guard(ctx->device);
  if (Aval_dev) IG_CK(ctx, launch_operator_csr(mesh->md, Aval_dev, ctx->stream), "copy A");
  if (M_dev)
    IG_CK(ctx, cudaMemcpyAsync(M_dev, mesh->md.M, sizeof(double) * mesh->n, cudaMemcpyDeviceToDevice, ctx->stream),
          "copy M");
  return IG_OK;
}

ig_status ig_operator32(ig_mesh* mesh, float* Aval_dev) {
  IG_NVTX("ig_operator32");
  if (!mesh || !Aval_dev) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (mesh->assembled < 2) {
    set_error(ctx, "FP32 operator requested before a mixed-precision assembly");
    return IG_ERR_STATE;
  }
  DeviceGuard guard(ctx->device);
  IG_CK(ctx, launch_operator32_csr(mesh->md, Aval_dev, ctx->stream), "copy A32");
  return IG_OK;
}

ig_status ig_solve(ig_mesh* mesh, const double* B_dev, int k, double* U_dev, const ig_solve_opts* opts,
                   ig_solve_info* info) {
  IG_NVTX("ig_solve");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled) {
    set_error(ctx, "solve before assemble");
    return IG_ERR_STATE;
  }
  if (!B_dev || !U_dev) return bad_arg(ctx, "B and U must be non-NULL");
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  if ((const void*)B_dev == (const void*)U_dev) return bad_arg(ctx, "B and U must not overlap");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  io->in[0] = B_dev;
  io->out[0] = U_dev;
  IG_CK(ctx, group_solve(mesh->group, k, mesh->assembled >= 2, *io, 1, o, ctx->stream), "solve");
  if (!info) return IG_OK;
  IG_CK(ctx, group_true_residual(mesh->group, k, *io, 1, ctx->stream), "residual");
  return collect_info(mesh, k, info);
}

ig_status ig_adjoint(ig_mesh* mesh, const double* V_dev, const double* B_dev, int b_is_V, const double* U_dev,
                     const double* G_dev, int k, double* gV_dev, double* gB_dev, double* gt_dev,
                     const ig_solve_opts* opts, ig_solve_info* info) {
  IG_NVTX("ig_adjoint");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled) {
    set_error(ctx, "adjoint before assemble");
    return IG_ERR_STATE;
  }
  if (!V_dev || !U_dev || !G_dev || !gV_dev) return bad_arg(ctx, "V, U, G and gV must be non-NULL");
  if (!b_is_V && !B_dev) return bad_arg(ctx, "B must be non-NULL unless b_is_V");
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  if (b_is_V && k != 3) return bad_arg(ctx, "b_is_V needs k == 3");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  io->in[0] = G_dev;
  io->out[0] = mesh->md.lam;
  IG_CK(ctx, group_solve(mesh->group, k, mesh->assembled >= 2, *io, 0, o, ctx->stream), "adjoint solve");
  CallDev call{};
  call.V = V_dev;
  call.B = b_is_V ? V_dev : B_dev;
  call.U = U_dev;
  call.gV = gV_dev;
  call.gB = gB_dev;
  call.gt = gt_dev;
  call.t = mesh->t;
  call.b_is_V = b_is_V ? 1 : 0;
  call.bstride = b_is_V ? 3 : k;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, launch_vjp(mesh->group, k, ctx->stream, 0, mesh->assembled == 3), "vjp");
  if (!info) return IG_OK;
  IG_CK(ctx, group_true_residual(mesh->group, k, *io, 0, ctx->stream), "residual");
  return collect_info(mesh, k, info);
}

ig_status ig_solve_begin(ig_mesh* mesh, const double* in_dev, int k, int rhs_mass, const ig_solve_opts* opts) {
  IG_NVTX("ig_solve_begin");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled) {
    set_error(ctx, "solve before assemble");
    return IG_ERR_STATE;
  }
  if (!in_dev) return bad_arg(ctx, "right-hand side is NULL");
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  io->in[0] = in_dev;
  io->out[0] = nullptr;
  IG_CK(ctx, group_begin(mesh->group, k, mesh->assembled >= 2, *io, rhs_mass ? 1 : 0, o, ctx->stream),
        "solve begin");
  return IG_OK;
}

ig_status ig_solve_end(ig_mesh* mesh, int k, double* out_dev, ig_solve_info* info) {
  IG_NVTX("ig_solve_end");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  DeviceGuard guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  io->in[0] = nullptr;
  io->out[0] = out_dev ? out_dev : mesh->md.lam;
  IG_CK(ctx, group_end(mesh->group, k, *io, ctx->stream), "solve end");
  if (!info) return IG_OK;
  return collect_info(mesh, k, info);
}

ig_status ig_vjp(ig_mesh* mesh, const double* V_dev, const double* B_dev, int b_is_V, const double* U_dev, int k,
                 double* gV_dev, double* gB_dev, double* gt_dev) {
  IG_NVTX("ig_vjp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled) {
    set_error(ctx, "gradient before assemble");
    return IG_ERR_STATE;
  }
  if (!V_dev || !U_dev || !gV_dev || (!b_is_V && !B_dev)) return bad_arg(ctx, "a required pointer is NULL");
  if (k < 1 || k > kMaxK || (b_is_V && k != 3)) return bad_arg(ctx, "bad k");
  DeviceGuard guard(ctx->device);
  CallDev call{};
  call.V = V_dev;
  call.B = b_is_V ? V_dev : B_dev;
  call.U = U_dev;
  call.gV = gV_dev;
  call.gB = gB_dev;
  call.gt = gt_dev;
  call.t = mesh->t;
  call.b_is_V = b_is_V ? 1 : 0;
  call.bstride = b_is_V ? 3 : k;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, launch_vjp(mesh->group, k, ctx->stream, 0, mesh->assembled == 3), "vjp");
  return IG_OK;
}

ig_status ig_mass_vjp(ig_mesh* mesh, const double* V_dev, const double* w_dev, double* gV_dev) {
  IG_NVTX("ig_mass_vjp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !w_dev || !gV_dev) return bad_arg(ctx, "V, w and gV must be non-NULL");
  DeviceGuard guard(ctx->device);
  CallDev call{};
  call.V = V_dev;
  call.gV = gV_dev;
  call.wm = w_dev;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, launch_vjp(mesh->group, 1, ctx->stream, 2), "mass vjp");
  return IG_OK;
}

ig_status ig_fairing_step(ig_mesh* mesh, double* V_dev, const double* T_dev, double t, double eta, int precision,
                          const ig_solve_opts* opts, double* loss_host, ig_solve_info* info3) {
  IG_NVTX("ig_fairing_step");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !T_dev) return bad_arg(ctx, "V and T must be non-NULL");
  if (!(eta >= 0.0) || !(eta < 1e300)) return bad_arg(ctx, "eta must be finite and >= 0");
  if (precision != IG_PRECISION_FP64 && precision != IG_PRECISION_MIXED)
    return bad_arg(ctx, "the fairing step runs in FP64 or mixed precision");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const size_t n = (size_t)mesh->n;
  if (!mesh->fair) IG_CK(ctx, mesh_alloc(mesh, &mesh->fair, 13 * n + 1), "alloc");
  double* U = mesh->fair;
  double* G = U + 3 * n;
  double* graw = G + 3 * n;
  double* gs = graw + 3 * n;
  double* w = gs + 3 * n;
  double* loss = w + n;
  ig_status st = ig_assemble(mesh, V_dev, t, precision);
  if (st != IG_OK) return st;
  const int mixed = mesh->assembled == 2;
  auto io = std::make_unique<IoTable>();
  auto solve = [&](const double* in, double* out, int rhs_mass, int slot) -> ig_status {
    io->in[0] = in;
    io->out[0] = out;
    IG_CK(ctx, group_solve(mesh->group, 3, mixed, *io, rhs_mass, o, ctx->stream), "solve");
    if (info3) {
      IG_CK(ctx, group_true_residual(mesh->group, 3, *io, rhs_mass, ctx->stream), "residual");
      ig_status s2 = collect_info(mesh, 3, &info3[slot]);
      if (s2 != IG_OK && s2 != IG_ERR_NOT_CONVERGED) return s2;
    }
    return IG_OK;
  };
  // forward: U = A^-1 M V
  if ((st = solve(V_dev, U, 1, 0)) != IG_OK) return st;
  // M-norm loss, its adjoint right-hand side G = M (U - T) and mass weights w = |U - T|^2 / 2
  IG_CK(ctx, launch_mnorm(mesh->group, U, T_dev, G, w, loss, ctx->stream), "loss");
  // adjoint: Lambda = A^-1 G, then dl/dV with B = V and the mass term of the loss
  if ((st = solve(G, mesh->md.lam, 0, 1)) != IG_OK) return st;
  CallDev call{};
  call.V = V_dev;
  call.B = V_dev;
  call.U = U;
  call.gV = graw;
  call.t = mesh->t;
  call.b_is_V = 1;
  call.bstride = 3;
  call.wm = w;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, launch_vjp(mesh->group, 3, ctx->stream, 1), "vjp");
  // Sobolev H^1 step with the same operator, then V <- V - eta g~
  if ((st = solve(graw, gs, 0, 2)) != IG_OK) return st;
  IG_CK(ctx, launch_step(V_dev, gs, eta, (long)(3 * n), ctx->num_sms, ctx->stream), "step");
  if (loss_host) {
    IG_CK(ctx, cudaMemcpyAsync(loss_host, loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "loss");
    IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  }
  return IG_OK;
}

ig_status ig_eigs(ig_mesh* mesh, int k, int iters, double* U_dev, double* lambda_host, const ig_solve_opts* opts,
                  ig_solve_info* info) {
  IG_NVTX("ig_eigs");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled || mesh->assembled == 3) {
    set_error(ctx, "eigs needs a mesh assembled in FP64 or mixed precision");
    return IG_ERR_STATE;
  }
  if (!U_dev) return bad_arg(ctx, "U must be non-NULL");
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  if (iters < 1) return bad_arg(ctx, "iters must be >= 1");
  if (!(mesh->t > 0.0)) return bad_arg(ctx, "the shift -1/t needs an assembled t > 0");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n;
  if (!mesh->eig) IG_CK(ctx, mesh_alloc(mesh, &mesh->eig, eig_workspace_doubles(n)), "alloc");
  double* Y = mesh->eig;
  IG_CK(ctx, eig_reset(mesh->eig, n, ctx->stream), "eigs");
  auto io = std::make_unique<IoTable>();
  io->in[0] = U_dev;
  io->out[0] = Y;
  const EigBuffers eb = eig_buffers(mesh->eig, n);
  auto io_warm = std::make_unique<IoTable>();
  io_warm->in[0] = eb.Yb;
  io_warm->out[0] = eb.X;
  for (int it = 0; it < iters; ++it) {
    // Y = (M + tL)^-1 M U, then U = Q(Y). After the first step the solve starts from
    // Y0 = U diag(R_cc) and finds the correction to the same accuracy relative to |M U|.
    if (it == 0) {
      IG_CK(ctx, group_solve(mesh->group, k, mesh->assembled == 2, *io, 1, o, ctx->stream), "eigs solve");
    } else {
      double ratio = 1.0;
      IG_CK(ctx, eig_warm(k, mesh->group.mds, mesh->eig, n, U_dev, &ratio, ctx->stream), "eigs");
      ig_solve_opts ow = o;
      ow.rel_tol = std::min(0.5, o.rel_tol * ratio);
      IG_CK(ctx, group_solve(mesh->group, k, mesh->assembled == 2, *io_warm, 0, ow, ctx->stream), "eigs solve");
      IG_CK(ctx, eig_addx(k, mesh->eig, n, ctx->stream), "eigs");
    }
    IG_CK(ctx, eig_step(k, mesh->eig, mesh->md.M, n, U_dev, ctx->stream), "eigs");
  }
  IG_CK(ctx, eig_finish(k, mesh->group.mds, mesh->t, mesh->eig, n, U_dev, ctx->stream), "eigs");
  if (!lambda_host && !info) return IG_OK;
  int fail = 0;
  IG_CK(ctx, eig_read(mesh->eig, n, k, lambda_host, &fail, ctx->stream), "eigs");
  if (info) {
    ig_status s = collect_info(mesh, k, info);  // the last solve's status and iterations
    if (s != IG_OK) return s;
  }
  if (fail) {
    set_error(ctx, "eigs: a Gram matrix was not positive definite (dependent or non-finite columns)");
    return IG_ERR_NONFINITE;
  }
  return IG_OK;
}

ig_status ig_eigs_vjp(ig_mesh* mesh, const double* V_dev, int k, int iters, const double* U_dev, const double* gU_dev,
                      double* gV_dev, const ig_solve_opts* opts) {
  IG_NVTX("ig_eigs_vjp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!mesh->assembled || mesh->assembled == 3) {
    set_error(ctx, "eigs_vjp needs a mesh assembled in FP64 or mixed precision");
    return IG_ERR_STATE;
  }
  if (!V_dev || !U_dev || !gU_dev || !gV_dev) return bad_arg(ctx, "V, U, gU and gV must be non-NULL");
  if (k < 1 || k > kMaxK) return bad_arg(ctx, "k must be in [1, 4]");
  if (iters < 1) return bad_arg(ctx, "iters must be >= 1");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n;
  if (!mesh->eig) IG_CK(ctx, mesh_alloc(mesh, &mesh->eig, eig_workspace_doubles(n)), "alloc");
  const EigBuffers eb = eig_buffers(mesh->eig, n);
  const int mixed = mesh->assembled == 2;
  IG_CK(ctx, eig_reset(mesh->eig, n, ctx->stream), "eigs_vjp");
  auto io = std::make_unique<IoTable>();
  auto solve = [&](const double* in, double* out, int rhs_mass) -> cudaError_t {
    io->in[0] = in;
    io->out[0] = out;
    return group_solve(mesh->group, k, mixed, *io, rhs_mass, o, ctx->stream);
  };
  // Y = (M + tL)^-1 M U*; R^-1 of Y^T M Y and the signs that map Y R^-1 onto U*; W = gU
  IG_CK(ctx, solve(U_dev, eb.Y, 1), "eigs_vjp solve");
  IG_CK(ctx, eig_vjp_prepare(k, mesh->eig, mesh->md.M, n, U_dev, gU_dev, ctx->stream), "eigs_vjp");
  // Neumann series of W = gU + J^T W, J^T W = M (M + tL)^-1 Ybar(W)
  for (int it = 0; it < iters; ++it) {
    IG_CK(ctx, eig_vjp_ybar(k, mesh->eig, mesh->md.M, n, ctx->stream), "eigs_vjp");
    IG_CK(ctx, solve(eb.Yb, eb.X, 0), "eigs_vjp solve");
    IG_CK(ctx, eig_vjp_next(k, mesh->eig, mesh->md.M, n, gU_dev, ctx->stream), "eigs_vjp");
  }
  // dl/dV = <Lambda, d(M U*)/dV - dA/dV Y> with Lambda = (M + tL)^-1 Ybar(W), plus the mass term
  // of the Gram matrix (weights -Y P Y^T)
  IG_CK(ctx, eig_vjp_ybar(k, mesh->eig, mesh->md.M, n, ctx->stream), "eigs_vjp");
  IG_CK(ctx, solve(eb.Yb, mesh->md.lam, 0), "eigs_vjp solve");
  IG_CK(ctx, eig_vjp_massw(k, mesh->eig, n, ctx->stream), "eigs_vjp");
  CallDev call{};
  call.V = V_dev;
  call.B = U_dev;
  call.U = eb.Y;
  call.gV = gV_dev;
  call.t = mesh->t;
  call.b_is_V = 0;
  call.bstride = k;
  call.wm = eb.wm;
  IG_CK(ctx, group_set_calls(mesh->group, &call, ctx->stream), "upload");
  IG_CK(ctx, launch_vjp(mesh->group, k, ctx->stream, 1), "vjp");
  int fail = 0;
  IG_CK(ctx, eig_read(mesh->eig, n, k, nullptr, &fail, ctx->stream), "eigs_vjp");
  if (fail) {
    set_error(ctx, "eigs_vjp: the Gram matrix of (M + tL)^-1 M U was not positive definite");
    return IG_ERR_NONFINITE;
  }
  return IG_OK;
}

// Shared set-up of the geodesic u-step and its gradient: argument checks, the source mask, the
// assembly at V with t = 1 and its rewrite into the source-constrained Laplacian.
static ig_status rgd_prepare(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, double rho,
                             double beta, int** src_out) {
  ig_ctx* ctx = mesh->ctx;
  if (mesh->md.clamp_on) {
    set_error(ctx, "the geodesic operator needs the plain cotangent Laplacian (L = D G): the cotangent clamp is on");
    return IG_ERR_STATE;
  }
  if (nsrc < 1) return bad_arg(ctx, "at least one source is needed (u_s = 0 fixes the constant)");
  if (!(rho >= 0.0) || !(beta >= 0.0) || !(rho + beta > 0.0) || !(rho + beta < 1e300))
    return bad_arg(ctx, "rho and beta must be finite, >= 0, and not both 0");
  const long n = (long)mesh->n;
  std::vector<int> mask((size_t)n, 0);
  for (int i = 0; i < nsrc; ++i) {
    if (sources_host[i] < 0 || sources_host[i] >= n) return bad_arg(ctx, "a source index is out of range");
    mask[(size_t)sources_host[i]] = 1;
  }
  if (!mesh->rgd) IG_CK(ctx, mesh_alloc(mesh, &mesh->rgd, 4 * (size_t)n + 8 + 3 * (size_t)mesh->m), "alloc");
  int* src = reinterpret_cast<int*>(mesh->rgd + n);
  IG_CK(ctx, cudaMemcpyAsync(src, mask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream), "sources");
  // the copy reads mask before this function returns
  IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "sources");
  ig_status st = ig_assemble(mesh, V_dev, 1.0, IG_PRECISION_FP64);
  if (st != IG_OK) return st;
  IG_CK(ctx, launch_rgd_operator(mesh->group.mds, (int)n, src, ctx->stream), "u-step operator");
  *src_out = src;
  return IG_OK;
}

ig_status ig_rgd_u_step(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, const double* y_dev,
                        const double* z_dev, double rho, double beta, double* u_dev, const ig_solve_opts* opts,
                        ig_solve_info* info) {
  IG_NVTX("ig_rgd_u_step");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !sources_host || !y_dev || !z_dev || !u_dev) return bad_arg(ctx, "V, sources, y, z and u must be non-NULL");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n;
  int* src = nullptr;
  ig_status st = rgd_prepare(mesh, V_dev, sources_host, nsrc, rho, beta, &src);
  if (st != IG_OK) return st;
  double* b = mesh->rgd;
  IG_CK(ctx, launch_rgd_rhs(mesh->group.mds, (int)n, V_dev, y_dev, z_dev, rho, beta, src, b, ctx->stream),
        "u-step rhs");
  auto io = std::make_unique<IoTable>();
  io->in[0] = b;
  io->out[0] = u_dev;
  cudaError_t e = group_solve(mesh->group, 1, 0, *io, 0, o, ctx->stream);
  if (e == cudaSuccess && info) e = group_true_residual(mesh->group, 1, *io, 0, ctx->stream);
  if (e == cudaSuccess && info) st = collect_info(mesh, 1, info);
  // the values are no longer the smoothing operator
  mesh->assembled = 0;
  IG_CK(ctx, e, "u-step solve");
  return st;
}

ig_status ig_rgd_u_step_vjp(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc,
                            const double* y_dev, const double* z_dev, double rho, double beta, const double* u_dev,
                            const double* gu_dev, double* gV_dev, double* gy_dev, double* gz_dev,
                            const ig_solve_opts* opts) {
  IG_NVTX("ig_rgd_u_step_vjp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !sources_host || !y_dev || !z_dev || !u_dev || !gu_dev || !gV_dev)
    return bad_arg(ctx, "V, sources, y, z, u, gu and gV must be non-NULL");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n;
  int* src = nullptr;
  ig_status st = rgd_prepare(mesh, V_dev, sources_host, nsrc, rho, beta, &src);
  if (st != IG_OK) return st;
  double* b = mesh->rgd;
  const double s = 1.0 / (beta + rho);
  // lam = L_D^-1 gu (zero on the sources), into the mesh's adjoint buffer
  IG_CK(ctx, launch_rgd_vec(gu_dev, src, (int)n, 0, 0.0, b, ctx->stream), "u-step adjoint rhs");
  auto io = std::make_unique<IoTable>();
  io->in[0] = b;
  io->out[0] = mesh->md.lam;
  cudaError_t e = group_solve(mesh->group, 1, 0, *io, 0, o, ctx->stream);
  if (e == cudaSuccess) e = launch_rgd_vec(u_dev, src, (int)n, 1, s, b, ctx->stream);  // B = u + s
  if (e == cudaSuccess) {
    // s <lam, dm> - <lam, dL u>: the smoothing step's VJP with t = 1, B = u + s, U = u
    CallDev call{};
    call.V = V_dev;
    call.B = b;
    call.U = u_dev;
    call.gV = gV_dev;
    call.t = 1.0;
    call.b_is_V = 0;
    call.bstride = 1;
    e = group_set_calls(mesh->group, &call, ctx->stream);
  }
  if (e == cudaSuccess) e = launch_vjp(mesh->group, 1, ctx->stream, 0);
  // s <lam, dD (rho z - y)>, and dl/dy, dl/dz
  if (e == cudaSuccess)
    e = launch_rgd_dD(mesh->group.mds, (int)n, (int)mesh->m, V_dev, y_dev, z_dev, rho, beta, gV_dev, gy_dev, gz_dev,
                      ctx->stream);
  mesh->assembled = 0;
  IG_CK(ctx, e, "u-step gradient");
  return IG_OK;
}

ig_status ig_rgd_admm(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, double rho, double beta,
                      double beta_k, int max_rounds, double tol, int adapt_rho, double* u_dev, double* y_dev,
                      double* z_dev, double* stats_host, const ig_solve_opts* opts) {
  IG_NVTX("ig_rgd_admm");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !sources_host || !u_dev || !y_dev || !z_dev) return bad_arg(ctx, "V, sources, u, y and z must be non-NULL");
  if (max_rounds < 1) return bad_arg(ctx, "max_rounds must be >= 1");
  if (!(rho > 0.0) || !(rho < 1e300) || !(beta_k >= 0.0) || !(beta_k <= 2.0))
    return bad_arg(ctx, "rho must be > 0 and finite, beta_k in [0, 2]");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return bad_arg(ctx, "tol must be finite and >= 0");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n, m = (long)mesh->m;
  int* src = nullptr;
  ig_status st = rgd_prepare(mesh, V_dev, sources_host, nsrc, rho, beta, &src);
  if (st != IG_OK) return st;
  // workspace: b [n], source mask [n], residual words (primal, dual), the warm-start ratio and the
  // worst solve status (8 doubles), z_old [m][3], the warm start's right-hand side [n] and correction [n]
  double* b = mesh->rgd;
  unsigned long long* res = reinterpret_cast<unsigned long long*>(mesh->rgd + 2 * n);  // primal, dual
  double* ratio_dev = mesh->rgd + 2 * n + 2;
  int* worst_dev = reinterpret_cast<int*>(mesh->rgd + 2 * n + 3);
  double* zold = mesh->rgd + 2 * n + 8;
  double* rhs_w = zold + 3 * m;
  double* delta = rhs_w + n;
  IoTable io, io_w;
  io.in[0] = b;
  io.out[0] = u_dev;
  io_w.in[0] = rhs_w;
  io_w.out[0] = delta;
  const bool watch = tol > 0.0 || adapt_rho != 0;  // residuals needed after every round
  double primal = 0.0, dual = 0.0;
  int rounds = 0, warm_skipped = 0;
  cudaError_t e = cudaMemsetAsync(worst_dev, 0, sizeof(int), ctx->stream);
  for (int it = 0; it < max_rounds && e == cudaSuccess; ++it) {
    e = launch_rgd_rhs(mesh->group.mds, (int)n, V_dev, y_dev, z_dev, rho, beta, src, b, ctx->stream);
    if (e == cudaSuccess && it == 0) {
      e = group_solve(mesh->group, 1, 0, io, 0, o, ctx->stream);
      if (e == cudaSuccess) e = launch_rgd_note_status(mesh->group.mds, worst_dev, ctx->stream);
    } else if (e == cudaSuccess) {
      // warm start from the last round's u: solve A d = b - A u for the correction, to the
      // tolerance that leaves |b - A (u + d)| <= rel_tol |b| (or skip it when u already meets it)
      double ratio = 0.0;
      e = launch_rgd_warm(mesh->group.mds, n, b, u_dev, rhs_w, ratio_dev, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&ratio, ratio_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e == cudaSuccess && !(ratio * o.rel_tol >= 1.0)) {
        ig_solve_opts ow = o;
        ow.rel_tol = o.rel_tol * ratio;
        e = group_solve(mesh->group, 1, 0, io_w, 0, ow, ctx->stream);
        if (e == cudaSuccess) e = launch_rgd_note_status(mesh->group.mds, worst_dev, ctx->stream);
        if (e == cudaSuccess) e = launch_rgd_axpy(u_dev, delta, n, ctx->stream);
      } else if (e == cudaSuccess) {
        ++warm_skipped;
      }
    }
    const bool need = watch || it == max_rounds - 1;
    if (e == cudaSuccess && need) e = cudaMemcpyAsync(zold, z_dev, sizeof(double) * 3 * m, cudaMemcpyDeviceToDevice,
                                                      ctx->stream);
    if (e == cudaSuccess && need) e = cudaMemsetAsync(res, 0, 2 * sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess)
      e = launch_rgd_zy(mesh->group.mds, (int)m, V_dev, u_dev, y_dev, z_dev, rho, beta_k, need ? res : nullptr,
                        ctx->stream);
    if (e == cudaSuccess && need) e = launch_rgd_dual(mesh->group.mds, (int)n, V_dev, z_dev, zold, src, rho, res + 1,
                                                      ctx->stream);
    rounds = it + 1;
    if (e != cudaSuccess || !watch) continue;
    unsigned long long bits[2] = {0, 0};
    e = cudaMemcpyAsync(bits, res, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    std::memcpy(&primal, &bits[0], sizeof(double));
    std::memcpy(&dual, &bits[1], sizeof(double));
    if (tol > 0.0 && primal <= tol && dual <= tol) break;
    // residual balancing: keep the primal and dual residuals within a factor of 10 of each other
    if (adapt_rho) {
      if (primal > 10.0 * dual) rho *= 2.0;
      else if (dual > 10.0 * primal) rho *= 0.5;
    }
  }
  mesh->assembled = 0;
  IG_CK(ctx, e, "admm");
  int worst = 0;
  IG_CK(ctx, cudaMemcpyAsync(&worst, worst_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "admm");
  if (stats_host && !watch) {
    unsigned long long bits[2] = {0, 0};
    IG_CK(ctx, cudaMemcpyAsync(bits, res, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream), "admm");
    IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "admm");
    std::memcpy(&primal, &bits[0], sizeof(double));
    std::memcpy(&dual, &bits[1], sizeof(double));
  }
  IG_CK(ctx, cudaStreamSynchronize(ctx->stream), "admm");
  if (stats_host) {
    stats_host[0] = rounds;
    stats_host[1] = primal;
    stats_host[2] = dual;
    stats_host[3] = rho;
    stats_host[4] = warm_skipped;
  }
  if (worst != IG_OK) {
    set_error(ctx, worst == IG_ERR_NOT_CONVERGED ? "a u-step solve reached max_iter above rel_tol"
                                                 : "a u-step solve met a non-finite value");
    return (ig_status)worst;
  }
  return IG_OK;
}

ig_status ig_rgd_admm_vjp(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, double rho,
                          double beta, double beta_k, const double* y_dev, const double* z_dev, const double* gu_dev,
                          int restart, int max_iter, double tol, double* gV_dev, double* w_dev, double* stats_host,
                          const ig_solve_opts* opts) {
  IG_NVTX("ig_rgd_admm_vjp");
  if (!mesh) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = mesh->ctx;
  if (!V_dev || !sources_host || !y_dev || !z_dev || !gu_dev || !gV_dev)
    return bad_arg(ctx, "V, sources, y, z, gu and gV must be non-NULL");
  if (!(rho > 0.0) || !(rho < 1e300) || !(beta_k >= 0.0) || !(beta_k <= 2.0))
    return bad_arg(ctx, "rho must be > 0 and finite, beta_k in [0, 2]");
  if (restart < 1 || restart > 100) return bad_arg(ctx, "restart must be in [1, 100]");
  if (max_iter < 1) return bad_arg(ctx, "max_iter must be >= 1");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return bad_arg(ctx, "tol must be finite and >= 0");
  const ig_solve_opts o = resolve_opts(opts);
  ig_status cs = check_opts(ctx, o);
  if (cs != IG_OK) return cs;
  DeviceGuard guard(ctx->device);
  const long n = (long)mesh->n, m = (long)mesh->m;
  int* src = nullptr;
  ig_status st = rgd_prepare(mesh, V_dev, sources_host, nsrc, rho, beta, &src);
  if (st != IG_OK) return st;
  double* b = mesh->rgd;
  const double s = 1.0 / (beta + rho);
  // workspace: u* [n], gbar [m][3], the right-hand side and (unless the caller takes it) w, [6m] each
  double* ws = nullptr;
  const size_t count = (size_t)n + 3 * (size_t)m + 6 * (size_t)m + (w_dev ? 0 : 6 * (size_t)m);
  IG_CK(ctx, cudaMalloc(&ws, sizeof(double) * count), "alloc");
  std::unique_ptr<double, void (*)(double*)> hold(ws, [](double* p) { cudaFree(p); });
  double* u = ws;
  double* gbar = u + n;
  double* rhs = gbar + 3 * m;
  double* w = w_dev ? w_dev : rhs + 6 * m;
  const MeshDev* mds = mesh->group.mds;
  auto io = std::make_unique<IoTable>();
  io->in[0] = b;
  auto solve_into = [&](double* out) -> cudaError_t {
    io->out[0] = out;
    return group_solve(mesh->group, 1, 0, *io, 0, o, ctx->stream);
  };
  // u* = the u-step at (y*, z*)
  cudaError_t e = launch_rgd_rhs(mds, (int)n, V_dev, y_dev, z_dev, rho, beta, src, b, ctx->stream);
  if (e == cudaSuccess) e = solve_into(u);
  // right-hand side (gy0, gz0): the u-step's VJP of gu, lam = L_D^-1 gu
  if (e == cudaSuccess) e = launch_rgd_vec(gu_dev, src, (int)n, 0, 0.0, b, ctx->stream);
  if (e == cudaSuccess) e = solve_into(mesh->md.lam);
  if (e == cudaSuccess) e = cudaMemsetAsync(rhs, 0, sizeof(double) * 6 * m, ctx->stream);
  if (e == cudaSuccess) e = launch_rgd_lamgrad(mds, (int)m, V_dev, -s, rho * s, rhs, ctx->stream);
  IG_CK(ctx, e, "admm adjoint set-up");
  // (I - J^T) v: the round's backward pass, with J^T's u-step part through one constrained solve
  auto apply = [&](const double* in, double* out) -> cudaError_t {
    cudaError_t e2 = launch_rgd_rvjp_face(mds, (int)m, V_dev, u, y_dev, in, rho, beta_k, gbar, out, ctx->stream);
    if (e2 == cudaSuccess) e2 = launch_rgd_gT(mds, (int)n, V_dev, gbar, nullptr, src, b, ctx->stream);
    if (e2 == cudaSuccess) e2 = solve_into(mesh->md.lam);
    if (e2 == cudaSuccess) e2 = launch_rgd_lamgrad(mds, (int)m, V_dev, s, -rho * s, out, ctx->stream);
    return e2;
  };
  GmresResult gr{};
  e = gmres_solve(apply, rhs, w, 6 * m, restart, max_iter, tol, ctx->stream, &gr);
  IG_CK(ctx, e, "admm adjoint GMRES");
  // dl/dV = the u-step's VJP of gu + G^T gbar(w), plus d<gbar(w), G u*>/dV
  e = launch_rgd_rvjp_face(mds, (int)m, V_dev, u, y_dev, w, rho, beta_k, gbar, nullptr, ctx->stream);
  if (e == cudaSuccess) e = launch_rgd_gT(mds, (int)n, V_dev, gbar, gu_dev, src, b, ctx->stream);
  if (e == cudaSuccess) e = solve_into(mesh->md.lam);
  if (e == cudaSuccess) e = launch_rgd_vec(u, src, (int)n, 1, s, b, ctx->stream);  // B = u + s
  if (e == cudaSuccess) {
    CallDev call{};
    call.V = V_dev;
    call.B = b;
    call.U = u;
    call.gV = gV_dev;
    call.t = 1.0;
    call.b_is_V = 0;
    call.bstride = 1;
    e = group_set_calls(mesh->group, &call, ctx->stream);
  }
  if (e == cudaSuccess) e = launch_vjp(mesh->group, 1, ctx->stream, 0);
  if (e == cudaSuccess)
    e = launch_rgd_dD(mds, (int)n, (int)m, V_dev, y_dev, z_dev, rho, beta, gV_dev, nullptr, nullptr, ctx->stream);
  if (e == cudaSuccess) e = launch_rgd_dG(mds, (int)n, (int)m, V_dev, u, gbar, gV_dev, ctx->stream);
  // the workspace is freed on return
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  mesh->assembled = 0;
  IG_CK(ctx, e, "admm adjoint gradient");
  if (stats_host) {
    stats_host[0] = gr.iterations;
    stats_host[1] = gr.rel_resid;
    stats_host[2] = gr.converged;
  }
  if (!std::isfinite(gr.rel_resid)) {
    set_error(ctx, "admm adjoint: GMRES produced a non-finite residual");
    return IG_ERR_NONFINITE;
  }
  if (!gr.converged) {
    set_error(ctx, "admm adjoint: GMRES reached max_iter above tol (the best iterate is used)");
    return IG_ERR_NOT_CONVERGED;
  }
  return IG_OK;
}

ig_status ig_profile_enable(int enable) {
  ProfState& P = prof_state();
  std::lock_guard<std::mutex> lk(P.mu);
  P.drain();
  P.acc.clear();
  P.on = enable != 0;
  return IG_OK;
}

int ig_profile_read(ig_kernel_stat* out, int max) {
  ProfState& P = prof_state();
  std::lock_guard<std::mutex> lk(P.mu);
  P.drain();
  int i = 0;
  for (auto& kv : P.acc) {
    if (out && i < max) {
      std::memset(&out[i], 0, sizeof(ig_kernel_stat));
      std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.first;
      out[i].total_ms = kv.second.second;
    }
    ++i;
  }
  return i;
}

}  // extern "C"
