// ig_internal.cuh -- shared definitions of the sm_103a implicit-smoothing library.
//
// Layout conventions on the device (all row-major, 32-bit indices):
//   F        [m][3]  int32      faces (copied at upload)
//   rowptr   [n+1]   int32      CSR row offsets of L / A (diagonal included, columns sorted)
//   col      [nnz]   int32      CSR columns
//   diagpos  [n]     int32      absolute index of the diagonal entry of each row
//   incptr   [n+1]   int32      vertex -> (face, corner) incidence offsets (3m entries)
//   inc      [3m]    int2       .x = face*4 + corner (sorted by face within a vertex),
//                               .y = slot of the edge to the next corner | slot of the edge
//                                    to the previous corner << 16 (slots relative to rowptr[v])
//   facew    [m][4]  double     per face: t*cot_c/2 for the three corners, area/3
//   sell_ptr [nslices+1] int32  sliced-ELL layout of the same pattern, slices of 32 rows: entry j
//   sell_col [nnz_sell] int32   of row r sits at sell_ptr[r/32] + 32 j + r%32 (column-major in the
//                               slice, so a warp's 32 rows read slot j with one contiguous load);
//                               rows shorter than the slice width are padded with value 0
//   A        [nnz_sell] double  A = M + t L in the sliced layout; A32 [nnz_sell] float (mixed)
//   M, Dinv  [n]     double     lumped mass and 1/A_ii;  Dinv32 [n] float
//   solver vectors x, r, q (and their FP32 copies, rhs): column-major [K][n] so that a warp's
//   accesses to consecutive rows are contiguous; p: [n][KP] (KP = 4 when K = 3) because it is
//   gathered by rows in the SpMV (one aligned 32-byte FP64 or 16-byte FP32 load per row)
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/iskra_gb300.h"

namespace ig {

constexpr int kBlock = 256;          // threads per CTA of every row- or face-parallel kernel
constexpr int kRowsPerThread = 4;    // rows per thread in the mixed-precision solver kernels
constexpr int kTileRows = kBlock * kRowsPerThread;  // one pass of the mixed-precision solver kernels
constexpr int kMaxTileRows32 = 64 * kTileRows;      // the largest mixed-precision tile (passes of kTileRows)
constexpr int kMaxPasses64 = 8;      // FP64 solver tiles: at most 8 passes of kBlock rows
constexpr int kTileRows64 = kBlock * kMaxPasses64;
constexpr int kMaxK = 4;
constexpr int kSmallTiles = 16;      // a single mesh of at most this many FP64 tiles loops in one cluster
constexpr int kPartStride = 8;       // doubles per tile in the partial-sum arrays

// Device error word bits (OR-ed by kernels, decoded on the host).
enum : int {
  kErrIndex = 1,
  kErrRepeated = 2,
  kErrUnused = 4,
  kErrValence = 8,
  kErrDegenerate = 16,
  kErrNonfinite = 32,
  kErrBounds = 64,  // bounds-checked build only: an index read from device data was out of range
};

// Bounds-checked build (compiled with -DIG_CHECK, a separate library): the indices the kernels
// read from device data (pattern columns, face vertices, incidence entries, row slots) are tested
// before use; one out of range sets kErrBounds in the mesh's error word and the access is skipped,
// so a corrupted structure is reported (as IG_ERR_INDEX_OUT_OF_RANGE by the next synchronising
// call) instead of faulting. The default build compiles the tests away.
__device__ __forceinline__ bool in_range_checked(long long i, long long size, int* err) {
  if (i >= 0 && i < size) return true;
  if (err) atomicOr(err, kErrBounds);
  return false;
}
#ifdef IG_CHECK
#define IG_IN_RANGE(i, size, errp) ::ig::in_range_checked((long long)(i), (long long)(size), (errp))
#else
#define IG_IN_RANGE(i, size, errp) true
#endif

// NVTX range around a C ABI call (visible in Nsight timelines; costs a function-pointer call
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define IG_NVTX(name) ::ig::NvtxRange ig_nvtx_range_(name)

// Solver state of one mesh, resident in device memory. The "last CTA" of each reduction
// (detected with a counter) writes the scalars; every other field is read-only for kernels.
struct SolveScal {
  double rz[kMaxK];      // r . z of the current iterate (inner iterate in mixed precision)
  double alpha[kMaxK];
  double beta[kMaxK];
  double bnorm2[kMaxK];  // ||rhs||^2 of the system being iterated
  double rhs2[kMaxK];    // ||rhs||^2 of the outer (FP64) system
  double relres[kMaxK];  // last relative residual seen by the stopping test
  double trueres[kMaxK]; // FP64 recomputed relative residual (filled on request)
  double scale[kMaxK];   // mixed precision: norm of the residual the inner system was scaled by
  int active[kMaxK];     // columns still iterating (the inner FP32 system in mixed precision)
  int active64[kMaxK];   // mixed precision: columns whose FP64 residual is still above tol
  double relres_inner[kMaxK];
  int inner_iter;        // mixed precision: iterations of the current inner solve
  int inner_cap;         // mixed precision: cap on iterations of one inner solve
  int k;
  int done;              // 1 once every column converged, failed or hit the cap
  int status;            // ig_status of this solve
  int iter;              // conjugate-gradient iterations so far
  int refine;            // mixed precision: refinements so far
  int phase;             // mixed precision: kPhaseInner / kPhaseApply / kPhaseRestart
  int max_iter, max_refine;
  double tol, inner_tol;
  unsigned int cnt[4];   // last-CTA counters (spmv, update, init/residual, vjp)
};

// Phases of a mixed-precision solve (per mesh).
enum : int {
  kPhaseInner = 0,    // FP32 conjugate-gradient iterations on A32 d = r32
  kPhaseApply = 1,    // x64 += scale * d, then the next spmv recomputes r64 = rhs - A64 x64
  kPhaseRestart = 2,  // r32 = r64 / scale, d = 0, new inner solve
};

// Everything a kernel needs about one mesh (plain device pointers, passed in device arrays so
// that a batch of meshes is a list of these).
struct MeshDev {
  int n, m, nnz, ntiles;   // ntiles = ceil(n / tile_rows)
  int tile_rows;           // rows per FP64 solver tile (<= kTileRows64, a multiple of 32), chosen at upload
  int ntiles32, tile_rows32;  // the same for the mixed-precision kernels (their own occupancy)
  int ntiles32u, tile_rows32u;  // the mixed-precision update's tiles (one wave on meshes of kBigRows or more)
  int nnz_sell;            // stored entries of the sliced layout (0: A is plain CSR on rowptr/col)
  int sell_w;              // every slice has this many entries per row (0: widths differ)
  const int* sell_ptr;     // [ceil(n/32)+1] slice offsets, or null for plain CSR
  const int* sell_col;     // [nnz_sell]
  // mixed precision: the columns as 16-bit offsets from each slice's first row, kept when every
  // stored column lies within +-32767 of its slice's first row (null otherwise); the FP32 SpMV
  // then reads these instead of sell_col
  const short* sell_c16;   // [nnz_sell] or null
  int k;
  double t;
  const int* F;
  const int* rowptr;
  const int* col;
  const int* diagpos;
  const int* incptr;
  const int2* inc;
  double* facew;
  double* A;
  float* A32;
  double* M;
  double* Dinv;
  float* Dinv32;
  // FP64 solver vectors: x, r, q [k][n]; p and z = D^-1 r [n][KP] (rows padded for the gathers)
  double* x;
  double* r;
  double* p;
  double* q;
  double* z;
  // mixed-precision inner vectors
  float* x32;
  float* r32;
  float* p32;
  float* q32;
  double* rhs;             // mixed precision: the outer right-hand side, kept for residuals
  // right-hand side of the outer system (caller buffer for the forward solve), and its mode
  const double* rhs_src;
  int rhs_mass;            // 1: rhs = M * rhs_src, 0: rhs = rhs_src
  double* lam;             // adjoint solution [n][k]
  double* gface;           // per-face gradient contributions [m][9]
  double* part;            // [ntiles][kPartStride] partial sums
  SolveScal* s;
  int* err;
  // FP32 face geometry (IG_PRECISION_MIXED_GEOM32): when geom32 is set the operator is the FP32
  // one in A32 (A is not formed; residuals read A32 exactly in FP64 arithmetic) and the face
  // kernels work on hi/lo float splits of the FP64 vectors (x = hi + lo, hi the first 24
  // significant bits of x, lo the rest rounded to float), so that differences of neighbouring
  // values keep FP32 relative accuracy.
  int geom32;
  float* vsplit;           // [n][8]: positions, hi (x, y, z, 0) then lo (x, y, z, 0)
  float* usplit;           // [n][8]: U, hi (k columns, padded to 4) then lo
  float* lsplit;           // [n][8]: Lambda, the same layout
  float* wv;               // [n]: <Lambda_v, B_v - U_v> per vertex
  // per-face weights [m][4] float and per-face gradients [m][9] float live in facew and gface
  // Cotangent clamp (ig_mesh_set_cot_clamp): when clamp_on, every corner's cotangent enters the
  // operator as max(cot, clamp_min), and a clamped corner adds nothing to dl/dV.
  int clamp_on;
  double clamp_min;
};

// Topology reads through the bounds checks of the checked build (plain loads otherwise): a bad
// value is reported in md.err and replaced by one that keeps the access inside its array.
// The incidence range of vertex v (within [0, 3m)):
__device__ __forceinline__ void inc_range(const MeshDev& md, int v, int& e0, int& e1) {
  e0 = __ldg(md.incptr + v);
  e1 = __ldg(md.incptr + v + 1);
#ifdef IG_CHECK
  if (!(e0 >= 0 && e0 <= e1 && e1 <= 3 * md.m)) {
    atomicOr(md.err, kErrBounds);
    e0 = e1 = 0;
  }
#endif
}
// Vertex c of face f (within [0, n)):
__device__ __forceinline__ int face_vertex(const MeshDev& md, int f, int c) {
  const int v = __ldg(md.F + 3 * f + c);
  return IG_IN_RANGE(v, md.n, md.err) ? v : 0;
}
// The face of an incidence entry (within [0, m)):
__device__ __forceinline__ int inc_face(const MeshDev& md, int fc) {
  const int f = fc >> 2;
  return IG_IN_RANGE(f, md.m, md.err) ? f : 0;
}

// Host-side helpers (ig_api.cu).
void set_error(ig_ctx* ctx, const std::string& msg);

// Kernel timing (process-wide, off by default): while profiling is on, every launch is
// bracketed by CUDA events on its stream and the device time is accumulated per kernel name.
bool prof_on();
struct ProfScope {
  int slot = -1;
  const char* name;
  cudaStream_t st;
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
};
#define IG_PROF(name, st) ::ig::ProfScope ig_prof_scope_((name), (st))

}  // namespace ig

// ---------------------------------------------------------------------------------------------
// Opaque types of the C ABI.
struct ig_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int solver_slots = 0;    // CTAs of the FP64 solver kernels resident at once on the device
  int solver_slots32 = 0;  // same for the mixed-precision solver kernels
  int live_meshes = 0;
  std::string last_error;
};

namespace ig {

// Loop control shared by every mesh of one launch group (a single mesh or a batch).
struct LoopCtl {
  unsigned int cnt;   // CTAs of the update kernel that have finished this iteration
  int iter;           // iterations of the device-side loop so far
  int cap;            // hard cap on iterations of the device-side loop
  int all_done;       // 1 once every mesh of the group is done
  int any_apply;      // mixed precision: some mesh will recompute its FP64 residual next
  int ndone_start;    // serving: meshes already done when the loop (re)started; the loop stops
                      // as soon as more are done (a whole solve sets it out of reach)
  // Active list: the meshes not yet done when it was last built, in mesh order. Meshes of at
  // least kBigRows rows are listed apart ("big"): every CTA takes their tiles cyclically (CTAs at
  // work at the same time then cover neighbouring rows, whose SpMV gathers share L2 lines). The
  // others get the offsets of their tiles in the FP64 and mixed tilings and are dealt in
  // contiguous chunks (a CTA changes mesh rarely) through per-CTA start tables. A finished mesh
  // costs nothing in later iterations. Rebuilt whenever more meshes are done.
  int nmesh;          // meshes of the group
  int nact;           // meshes in the chunked list
  int nbig;           // meshes in the big list
  int ndone_list;     // meshes done when the list was built
  int grid64, grid32; // grids of the loop kernels (the start tables have one entry per CTA)
  int napp_big;       // big meshes in the Apply list
  int* act_mesh;      // [nmesh]
  int* act_off64;     // [nmesh + 1]
  int* act_off32;     // [nmesh + 1]
  int* big_mesh;      // [nmesh]
  int4* start64;      // [grid64]: each CTA's (list position, local tile, mesh, tile count)
  int4* start32;      // [grid32]
  // Mixed precision: the meshes about to recompute their FP64 residual (Apply phase), listed
  // the same way (mixed tiling only); rebuilt in every iteration that has any.
  int* app_mesh;      // [nmesh]
  int* app_off32;     // [nmesh + 1]
  int* app_big;       // [nmesh]
  int4* app_start32;  // [grid32]
};

constexpr int kBigRows = 1 << 20;

// What a loop kernel walks: a chunked list with its start table and a big list with its count.
struct ListRef {
  const int4* start;
  const int* act;
  const int* big;
  const int* nbig;
};

// Per-launch pointers that change from call to call (kept out of the cached graphs).
constexpr int kMaxIo = 1024;
struct IoTable {
  const double* in[kMaxIo];
  double* out[kMaxIo];
};

// Per-call arguments of one mesh for the assembly and gradient kernels (caller buffers change
// from call to call; they reach the kernels through this small device table).
struct CallDev {
  const double* V;   // positions [n][3]
  const double* B;   // right-hand side [n][k] (or V when b_is_V)
  const double* U;   // forward solution [n][k]
  double* gV;        // dl/dV [n][3]
  double* gB;        // dl/dB [n][k] or null
  double* gt;        // dl/dt (one double) or null
  double t;          // time step of the assembled operator
  int b_is_V;
  int bstride;       // columns of B (3 when b_is_V)
  const double* wm;  // per-vertex weights w [n] of the mass term d(sum_i M_i(V) w_i)/dV (VJP
                     // modes 1 and 2; see launch_vjp)
};

// A cached solver launch for one (k, precision): a CUDA graph whose WHILE node runs the
// iteration body until the device sets the loop condition to 0.
struct SolvePlan {
  int k = 0;
  int mixed = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// A group of meshes solved by the same kernel launches (a single mesh is a group of one).
struct Group {
  int nmesh = 0;
  int ntiles = 0;                 // total tiles over all meshes
  MeshDev* mds = nullptr;         // device array [nmesh]
  int2* tiles = nullptr;          // device array [ntiles]: (mesh, local tile)
  int ntiles32 = 0;
  int2* tiles32 = nullptr;        // the tiling of the mixed-precision kernels
  int grid64 = 0, grid32 = 0;     // persistent grid of the loop kernels: min(tiles, resident slots)
  int* flags_dev = nullptr;       // [nmesh] done flags gathered for the host (serving)
  LoopCtl* ctl = nullptr;         // device
  int* act_buf = nullptr;         // device storage of the active list and start tables (LoopCtl)
  ListRef list64{}, list32{}, listapp{};  // what the FP64, mixed and residual loop kernels walk
  int* done_host = nullptr;       // pinned host word for the host-driven loop
  SolvePlan plans[2][kMaxK + 1];  // [mixed][k]
  cudaStream_t capture_stream = nullptr;
  // 256-element tiles for the face- and row-parallel kernels: (mesh, local tile)
  int nface_tiles = 0, nrow_tiles = 0;
  int2* face_tiles = nullptr;
  int2* row_tiles = nullptr;
  CallDev* calls_dev = nullptr;   // [nmesh]
  CallDev* calls_host = nullptr;  // pinned staging for calls_dev
  cudaEvent_t calls_ev = nullptr; // the last upload of calls_host has been read
  std::vector<MeshDev> host_mds;  // host copy of mds
};

// Does some mesh of the group clamp its cotangents (host copy of the descriptors)?
inline bool group_any_clamp(const Group& g) {
  for (const MeshDev& md : g.host_mds)
    if (md.clamp_on) return true;
  return false;
}
cudaError_t group_init(Group& g, const MeshDev* host_mds, int nmesh, int slots64, int slots32, cudaStream_t st);
cudaError_t group_upload_mds(Group& g, cudaStream_t st);
cudaError_t group_set_calls(Group& g, const CallDev* calls, cudaStream_t st);
void group_destroy(Group& g);
cudaError_t group_solve(Group& g, int k, int mixed, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                        cudaStream_t st);
cudaError_t group_true_residual(Group& g, int k, const IoTable& io, int rhs_mass, cudaStream_t st);
cudaError_t mesh_ensure_mixed(ig_mesh* mesh, cudaStream_t st);
cudaError_t mesh_ensure_geom32(ig_mesh* mesh, cudaStream_t st);
cudaError_t mesh_set_geom32(ig_mesh* mesh, int geom32, cudaStream_t st);
int solver_blocks_per_sm();        // ig_pcg.cu: min resident CTAs per SM of the FP64 loop kernels
int solver_blocks_per_sm_mixed();  // ig_pcg_mixed.cu: same for the mixed-precision loop kernels
cudaError_t group_solve_mixed(Group& g, int k, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                              cudaStream_t st);
// Serving: start a solve (init), advance a group's running solves by a bounded number of
// iterations (stopping early once a running member finishes; done flags to the host), and write
// a finished solve's result.
cudaError_t group_begin(Group& g, int k, int mixed, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                        cudaStream_t st);
cudaError_t group_begin_mixed(Group& g, int k, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                              cudaStream_t st);
cudaError_t group_iterate(Group& g, int k, int mixed, int budget, int* done_host, cudaStream_t st);
cudaError_t group_host_loop_mixed(Group& g, int k, int budget, cudaStream_t st);
cudaError_t group_end(Group& g, int k, const IoTable& io, cudaStream_t st);

}  // namespace ig

// A mesh: topology, operator, solver workspace and its own launch group.
struct ig_mesh {
  ig_ctx* ctx = nullptr;
  int64_t n = 0, m = 0, nnz = 0;
  int64_t bytes = 0;
  int assembled = 0;        // 0 none, 1 FP64, 2 mixed, 3 mixed with FP32 face geometry
  double t = 0.0;
  int ws_k = 0;             // solver vectors allocated for this many columns
  ig::MeshDev md{};         // host copy of the device pointers
  ig::Group group;          // this mesh alone
  std::vector<void*> allocs;
  double* fair = nullptr;   // inverse-fairing workspace: U, G, g, g~ [n][3], w [n], loss (on first use)
  double* eig = nullptr;    // eigen-iteration workspace (eig_workspace_doubles, on first use)
  double* rgd = nullptr;    // geodesic workspace: right-hand side [n], source mask [n] ints, scalars [8],
                            // previous z [m][3]
};

// ---------------------------------------------------------------------------------------------
// Kernel launchers (each file defines its own).
namespace ig {

// ig_pattern.cu
cudaError_t exclusive_scan_int(const int* in, int* out, int count, int* total_out_dev, int* scratch,
                               size_t scratch_ints, cudaStream_t st);
size_t scan_scratch_ints(int count);
cudaError_t launch_pattern_count(const int* F, int m, int n, int* deg, int* err, cudaStream_t st);
cudaError_t launch_pattern_fill(const int* F, int m, const int* incptr, int* fill, int* inc_fc, cudaStream_t st);
cudaError_t launch_pattern_rows(const int* F, int n, const int* incptr, int* inc_fc, int* nbr, int* rowlen,
                                int* err, cudaStream_t st);
cudaError_t launch_pattern_cols(const int* F, int n, const int* incptr, const int* inc_fc, const int* nbr,
                                const int* rowptr, int* col, int* diagpos, int2* inc, int* err, cudaStream_t st);
cudaError_t launch_sell_width(const int* rowptr, int n, int* width32, cudaStream_t st);
cudaError_t launch_sell_c16(const int* sell_ptr, const int* sell_col, int n, short* c16, int* nfar,
                            cudaStream_t st);
cudaError_t launch_sell_fill(const int* rowptr, const int* col, int n, const int* sell_ptr, int* sell_col,
                             cudaStream_t st);

// ig_assemble.cu (per-call V and t come from g.calls_dev); mode: 0 FP64, 1 mixed (FP64 geometry
// and operator, FP32 copy), 2 mixed with FP32 face geometry (FP32 operator only)
cudaError_t launch_assemble(Group& g, int mode, cudaStream_t st);
cudaError_t launch_operator_csr(const MeshDev& md, double* Acsr, cudaStream_t st);
cudaError_t launch_operator32_csr(const MeshDev& md, float* Acsr, cudaStream_t st);

// ig_pcg.cu: see Group above

// ig_eigs.cu: shift-invert subspace iteration (workspace of eig_workspace_doubles(n) doubles)
size_t eig_workspace_doubles(long n);
cudaError_t eig_reset(double* ws, long n, cudaStream_t st);
// Q of one step: Y (the workspace's first [n][k]) -> U = Y R^-1
cudaError_t eig_step(int k, double* ws, const double* M, long n, double* U, cudaStream_t st);
// canonical signs of U's columns and the eigenvalues (u^T A u - u^T M u) / t
cudaError_t eig_finish(int k, const MeshDev* mds, double t, double* ws, long n, double* U, cudaStream_t st);
cudaError_t eig_read(double* ws, long n, int k, double* lambda_host, int* fail_host, cudaStream_t st);
// warm start of a step after the first: Y = U diag(R_cc of the last step), Ybar = M U - A Y, and
// (synchronising) min_c |M U_c| / |Ybar_c| into *tol_ratio_host; then, after solving A X = Ybar,
// eig_addx: Y += X
cudaError_t eig_warm(int k, const MeshDev* mds, double* ws, long n, const double* U, double* tol_ratio_host,
                     cudaStream_t st);
cudaError_t eig_addx(int k, double* ws, long n, cudaStream_t st);
// gradient through the fixed point: Y (= (M + tL)^-1 M U*) must be in the workspace first
struct EigBuffers {
  double *Y, *Yb, *X, *W, *wm;  // Y, Ybar, the solve of Ybar, the Neumann iterate W, mass weights
};
EigBuffers eig_buffers(double* ws, long n);
cudaError_t eig_vjp_prepare(int k, double* ws, const double* M, long n, const double* U, const double* gU,
                            cudaStream_t st);                      // R^-1, signs, W = gU
cudaError_t eig_vjp_ybar(int k, double* ws, const double* M, long n, cudaStream_t st);  // P, Ybar from W
cudaError_t eig_vjp_next(int k, double* ws, const double* M, long n, const double* gU, cudaStream_t st);  // W = gU + M X
cudaError_t eig_vjp_massw(int k, double* ws, long n, cudaStream_t st);  // wm = -Y P Y^T per row

// ig_rgd.cu: the u-step of the regularized-geodesic ADMM (mds: a group of one mesh)
cudaError_t launch_rgd_operator(const MeshDev* mds, int n, const int* src, cudaStream_t st);
cudaError_t launch_rgd_rhs(const MeshDev* mds, int n, const double* V, const double* y, const double* z, double rho,
                           double beta, const int* src, double* b, cudaStream_t st);
// warm start of a u-step solve: rhs = b - A u and *ratio = |b| / |rhs| (device scalar)
cudaError_t launch_rgd_warm(const MeshDev* mds, long n, const double* b, const double* u, double* rhs, double* ratio,
                            cudaStream_t st);
cudaError_t launch_rgd_axpy(double* u, const double* d, long n, cudaStream_t st);  // u += d
// *worst = max(*worst, status of the mesh's last solve)
cudaError_t launch_rgd_note_status(const MeshDev* mds, int* worst, cudaStream_t st);
// out = x with zeros on the sources (add_s = 0), or x + s (add_s = 1)
cudaError_t launch_rgd_vec(const double* x, const int* src, int n, int add_s, double s, double* out, cudaStream_t st);
// one ADMM z-step and dual step per face (primal: max_f |G u - z| as double bits, may be null)
cudaError_t launch_rgd_zy(const MeshDev* mds, int m, const double* V, const double* u, double* y, double* z, double rho,
                          double beta_k, unsigned long long* primal, cudaStream_t st);
// dual residual rho max_i |(D (z - zold))_i| / m_i over non-source vertices, as double bits
cudaError_t launch_rgd_dual(const MeshDev* mds, int n, const double* V, const double* z, const double* zold,
                            const int* src, double rho, unsigned long long* dual, cudaStream_t st);
// the divergence term of dl/dV (added to gV) and dl/dy, dl/dz (may be null), with lam in md.lam
cudaError_t launch_rgd_dD(const MeshDev* mds, int n, int m, const double* V, const double* y, const double* z,
                          double rho, double beta, double* gV, double* gy, double* gz, cudaStream_t st);
// the fixed-point adjoint of the rounds: per face abar, gbar and (when out is given) the face parts of
// (I - J^T) w, for w and out laid out [wy (m x 3) | wz (m x 3)]
cudaError_t launch_rgd_rvjp_face(const MeshDev* mds, int m, const double* V, const double* u, const double* y,
                                 const double* w, double rho, double beta_k, double* gbar, double* out,
                                 cudaStream_t st);
// ubar = G^T gbar (+ add when given), 0 on the sources
cudaError_t launch_rgd_gT(const MeshDev* mds, int n, const double* V, const double* gbar, const double* add,
                          const int* src, double* ubar, cudaStream_t st);
// out_y += cy area grad(lam), out_z += cz area grad(lam), with lam in md.lam
cudaError_t launch_rgd_lamgrad(const MeshDev* mds, int m, const double* V, double cy, double cz, double* out,
                               cudaStream_t st);
// gV += d<W, G u>/dV at fixed u and W (through md.gface)
cudaError_t launch_rgd_dG(const MeshDev* mds, int n, int m, const double* V, const double* u, const double* W,
                          double* gV, cudaStream_t st);

// ig_gmres.cu: restarted GMRES on device vectors (deterministic reductions), for the fixed-point
// adjoint; apply(in, out) computes out = A in on the stream
struct GmresResult {
  int iterations;    // Arnoldi steps taken (one product with A each, plus one per restart)
  double rel_resid;  // the final residual estimate relative to |rhs|
  int converged;
};
cudaError_t gmres_solve(const std::function<cudaError_t(const double*, double*)>& apply, const double* rhs, double* x,
                        long N, int restart, int max_iter, double rel_tol, cudaStream_t st, GmresResult* res);

// ig_vjp.cu
// mode 0: solve terms; 1: solve terms and the mass weights of the calls; 2: mass weights alone.
// geom32: the group was assembled with FP32 face geometry; mode 0 then runs the FP32 per-face
// gradient (FP64 for near-degenerate faces), the other modes the FP64 one.
cudaError_t launch_vjp(Group& g, int k, cudaStream_t st, int mode = 0, int geom32 = 0);
// ig_fairing.cu
cudaError_t launch_mnorm(Group& g, const double* U, const double* T, double* G, double* w, double* loss,
                         cudaStream_t st);
cudaError_t launch_step(double* V, const double* g, double eta, long count, int num_sms, cudaStream_t st);

}  // namespace ig
