// Host driver and C ABI (include/opt_gb300.h): problem planning, the GN and
// LM outer loops (Sec. 4), CUDA-graph replay of a whole solve, and the parity
// hooks (evalJTF, applyJTJ, evalF of Sec. 4.2).
//
// A solve is one fixed sequence of stream-ordered launches: copy x in, reset
// the device scalars, then per outer iteration PCGInit, `inner` x (applyJTJ,
// vector update), and the outer update (GN: x += delta; LM: trial energy,
// gain-ratio decision, conditional x += delta), then the final energy and the
// copy of x out.  Every decision (PCG breakdown, LM accept / reject, LM
// convergence) is taken on the device and read by later kernels, so the
// sequence never needs the host and is captured once as a CUDA graph.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"
#include "opt_launch.h"
#include "opt_problem.h"

using namespace optgb;

namespace {
thread_local std::string g_err;
}  // namespace

// Records the failed call for opt_last_error and clears the sticky error.
opt_status optgb::cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? OPT_ERR_OOM : OPT_ERR_CUDA;
}

namespace {

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

#define CKS(call)                          \
  do {                                     \
    opt_status s_ = (call);                \
    if (s_ != OPT_OK) return s_;           \
  } while (0)

__global__ void k_reset(Scalars* s, int n, double lambda0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) scalars_reset(s + i, lambda0);
}

__global__ void k_force_active(Scalars* s, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  s[i].pcg_active = 1;
  s[i].done = 0;
}

// LM decision (Sec. 4; Nielsen's damping update), one thread per problem.
__global__ void k_lm_decide(Scalars* s, int n, double eta, double lmin, double lmax, double rel_tol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lm_decide(s + i, eta, lmin, lmax, rel_tol);
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Locality order of graph vertices: ascending Morton (Z-order) code of the
// rest positions quantised to 10 bits per axis inside their bounding box,
// ties by caller index.  Neighbouring vertices of a surface mesh end up close
// in memory, so the gather kernels find most neighbour records in cache.
std::vector<int> morton_order(const std::vector<float>* U, int V) {
  float lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = hi[c] = V ? U[c][0] : 0.f;
    for (int v = 1; v < V; ++v) {
      lo[c] = std::min(lo[c], U[c][v]);
      hi[c] = std::max(hi[c], U[c][v]);
    }
  }
  auto spread = [](uint32_t x) {   // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
  };
  std::vector<uint32_t> code((size_t)V);
  for (int v = 0; v < V; ++v) {
    uint32_t cv = 0;
    for (int c = 0; c < 3; ++c) {
      const float ext = hi[c] - lo[c];
      const float t = ext > 0.f ? (U[c][v] - lo[c]) / ext : 0.f;
      const uint32_t qv = (uint32_t)std::min(1023.f, std::max(0.f, t * 1023.f));
      cv |= spread(qv) << c;
    }
    code[v] = cv;
  }
  // stable least-significant-digit radix sort of the 30-bit codes (3 x 10
  // bits): equal codes keep the caller order
  std::vector<int> perm((size_t)V), tmp((size_t)V);
  for (int v = 0; v < V; ++v) perm[v] = v;
  for (int pass = 0; pass < 3; ++pass) {
    const int shift = 10 * pass;
    std::vector<int> cnt(1025, 0);
    for (int v = 0; v < V; ++v) cnt[((code[perm[v]] >> shift) & 1023u) + 1] += 1;
    for (int b = 0; b < 1024; ++b) cnt[b + 1] += cnt[b];
    for (int v = 0; v < V; ++v) tmp[(size_t)cnt[(code[perm[v]] >> shift) & 1023u]++] = perm[v];
    perm.swap(tmp);
  }
  return perm;
}

}  // namespace


namespace {

// Problem memory comes from a library-owned stream-ordered pool per device
// that keeps freed blocks: planning and tearing down problems (the server
// does both continuously) then neither goes back to the driver nor waits for
// the device.  nullptr if the pool cannot be made (plain cudaMalloc then).
cudaMemPool_t problem_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[128] = {};
  static bool failed[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev] && !failed[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
      pools[dev] = nullptr;
      failed[dev] = true;
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return pools[dev];
}

// Zero-filled device array owned by the problem (ordered on the legacy
// stream; planning ends with a synchronising copy before any other stream
// touches it).
template <class T>
opt_status dalloc(opt_problem* pb, T** ptr, size_t n) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  cudaMemPool_t pool = problem_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, nullptr) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "device allocation");
  pb->allocs.push_back(p);
  pb->pooled.push_back(pool != nullptr);
  e = cudaMemsetAsync(p, 0, bytes, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  *ptr = static_cast<T*>(p);
  return OPT_OK;
}

template <class T>
opt_status upload(T* dst, const std::vector<T>& src) {
  if (src.empty()) return OPT_OK;
  CK(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return OPT_OK;
}

template <class T>
opt_status download(std::vector<T>& dst, const T* src, size_t n) {
  dst.resize(n);
  if (n == 0) return OPT_OK;
  CK(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
  return OPT_OK;
}

bool all_finite(const std::vector<float>& v) {
  for (float f : v)
    if (!std::isfinite(f)) return false;
  return true;
}

bool is_grid(const opt_problem* pb) { return pb->kind == K_WARP || pb->kind == K_POISSON; }

// distinct-diagonal plane of unknown component c
int mplane_of(int kind, int c) {
  if (kind == K_WARP || kind == K_WARPG) return c == 2 ? 1 : 0;   // K_MESH / K_VOLUME below
  if (kind == K_POISSON) return 0;
  return c < 3 ? 0 : c - 2;
}

opt_status common_setup(opt_problem* pb) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&pb->sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaStreamCreateWithFlags(&pb->cap_stream, cudaStreamNonBlocking));
  CK(cudaEventCreate(&pb->ev0));
  CK(cudaEventCreate(&pb->ev1));
  CKS(dalloc(pb, &pb->d_s, 1));
  return OPT_OK;
}

// Graph problems keep their vertices in a locality order (internal vertex k
// is the caller's vertex perm[k]); these move one plane between the orders.
__global__ void k_gather_vertices(float* __restrict__ dst, const float* __restrict__ src, const int* __restrict__ perm,
                                  int V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < V) dst[k] = src[perm[k]];
}
__global__ void k_scatter_vertices(float* __restrict__ dst, const float* __restrict__ src,
                                   const int* __restrict__ perm, int V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < V) dst[perm[k]] = src[k];
}

}  // namespace

namespace optgb {

// copy between caller dense planes (caller order) and internal planes
// (pitched rows for grids, locality order for graphs)
opt_status copy_planes_in(const opt_problem* pb, float* internal, float* const* user, int n,
                          cudaStream_t st) {
  for (int c = 0; c < n; ++c) {
    if (is_grid(pb)) {
      CK(cudaMemcpy2DAsync(internal + c * pb->plane, (size_t)pb->P * 4, user[c], (size_t)pb->W * 4,
                           (size_t)pb->W * 4, pb->H, cudaMemcpyDeviceToDevice, st));
    } else {
      k_gather_vertices<<<(pb->V + 255) / 256, 256, 0, st>>>(internal + c * pb->plane, user[c], pb->d_perm, pb->V);
      CK(cudaGetLastError());
    }
  }
  return OPT_OK;
}
opt_status copy_planes_out(const opt_problem* pb, float* const* user, const float* internal, int n,
                           cudaStream_t st) {
  for (int c = 0; c < n; ++c) {
    if (is_grid(pb)) {
      CK(cudaMemcpy2DAsync(user[c], (size_t)pb->W * 4, internal + c * pb->plane, (size_t)pb->P * 4,
                           (size_t)pb->W * 4, pb->H, cudaMemcpyDeviceToDevice, st));
    } else {
      k_scatter_vertices<<<(pb->V + 255) / 256, 256, 0, st>>>(user[c], internal + c * pb->plane, pb->d_perm, pb->V);
      CK(cudaGetLastError());
    }
  }
  return OPT_OK;
}

}  // namespace optgb

namespace {

void dense_planes(const opt_problem* pb, const float* base, float** out, int n) {
  for (int c = 0; c < n; ++c) out[c] = const_cast<float*>(base) + c * pb->ulen;
}

GridLaunch grid_launch(const opt_problem* pb, cudaStream_t st) {
  return GridLaunch{pb->dg, pb->d_chunks, pb->d_tiles, pb->d_part, pb->nchunks, st, pb->hg.tw,
                    pb->hg.mask != nullptr};
}
MeshLaunch mesh_launch(const opt_problem* pb, cudaStream_t st) {
  return MeshLaunch{pb->dm, pb->d_vchunks, pb->d_echunks, pb->d_part, pb->nvchunks,
                    pb->nechunks, st, pb->kind == K_WARPG ? 2 : (pb->kind == K_EMBED ? 12 : 3),
                    pb->kind == K_VOLUME ? 1 : 0, pb->apply_form ? pb->d_tchunks : nullptr, pb->ntchunks};
}

opt_status upload_desc(opt_problem* pb, cudaStream_t st) {
  if (is_grid(pb))
    CK(cudaMemcpyAsync(pb->dg, &pb->hg, sizeof(GridProb), cudaMemcpyHostToDevice, st));
  else
    CK(cudaMemcpyAsync(pb->dm, &pb->hm, sizeof(MeshProb), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return OPT_OK;
}

void set_flags(opt_problem* pb, int lm, int use_precond, double* ehist) {
  if (is_grid(pb)) {
    pb->hg.lm = lm;
    pb->hg.use_precond = use_precond;
    pb->hg.Ehist = ehist;
  } else {
    pb->hm.lm = lm;
    pb->hm.use_precond = use_precond;
    pb->hm.Ehist = ehist;
  }
}

// --- stage launchers (dispatch on the domain) ------------------------------
bool wide_warp(const opt_problem* pb) { return pb->kind == K_WARP && pb->hg.csn != nullptr; }

// csn_in: a wide warp's PCGInit reads cos / sin of theta written by the
// previous outer update (or launch_grid_csn)
void st_init(opt_problem* pb, cudaStream_t st, int k, float dmin, float dmax, int csn_in = 0) {
  if (is_grid(pb)) launch_grid_init(pb->kind, grid_launch(pb, st), k, dmin, dmax, csn_in);
  else launch_mesh_init(mesh_launch(pb, st), k, dmin, dmax);
}
void st_apply(opt_problem* pb, cudaStream_t st, const float* pov, int par, int update) {
  if (is_grid(pb)) launch_grid_apply(pb->kind, grid_launch(pb, st), pov, par, update);
  else launch_mesh_apply(mesh_launch(pb, st), pov, par, update);
}
void st_update(opt_problem* pb, cudaStream_t st, int par) {
  if (is_grid(pb)) launch_grid_update(pb->kind, grid_launch(pb, st), par);
  else launch_mesh_update(mesh_launch(pb, st), par);
}
void st_energy(opt_problem* pb, cudaStream_t st, int mode, int hist_idx) {
  if (is_grid(pb)) launch_grid_energy(pb->kind, grid_launch(pb, st), mode, hist_idx);
  else launch_mesh_energy(mesh_launch(pb, st), mode, hist_idx);
}
// csn_out: a wide warp's update also writes cos / sin of the new theta
void st_step(opt_problem* pb, cudaStream_t st, int cond, int csn_out = 0) {
  if (is_grid(pb)) launch_grid_step(pb->kind, grid_launch(pb, st), cond, csn_out);
  else launch_mesh_step(mesh_launch(pb, st), cond);
}

opt_status check_params(const opt_solve_params& p, bool lm) {
  if (p.outer < 1 || p.inner < 0 || p.outer > (1 << 20) || p.inner > (1 << 20)) return OPT_ERR_INVALID_ARG;
  if (p.use_precond != 0 && p.use_precond != 1) return OPT_ERR_INVALID_ARG;
  if (lm) {
    if (!(p.lambda0 >= 0.0) || !std::isfinite(p.lambda0)) return OPT_ERR_INVALID_ARG;
    if (!(p.lambda_min >= 0.0) || !(p.lambda_min <= p.lambda_max)) return OPT_ERR_INVALID_ARG;
    if (!(p.diag_min >= 0.0) || !(p.diag_min <= p.diag_max)) return OPT_ERR_INVALID_ARG;
    if (!std::isfinite(p.eta) || !(p.rel_tol >= 0.0)) return OPT_ERR_INVALID_ARG;
  }
  return OPT_OK;
}

// The whole solve as stream-ordered work (captured into a graph or run directly).
// The PCG loop runs as one cooperative launch per outer iteration when asked
// for, matrix-free, on wide warp tiles, and every chunk's block fits on the
// device at once.
bool use_persistent(const opt_problem* pb, const opt_solve_params& p) {
  return p.persistent && !p.materialized && p.inner > 0 && pb->d_gbar && pb->nchunks <= pb->coop_cap;
}

// The single-reduction PCG iteration runs where asked for on warps and
// Poisson problems planned with 128-pixel tiles (they have z / w buffers),
// matrix-free; elsewhere the two-pass form.
bool use_fused(const opt_problem* pb, const opt_solve_params& p) {
  return p.pcg_form == 1 && !p.materialized && (pb->kind == K_WARP || pb->kind == K_POISSON) &&
         pb->hg.zb != nullptr;
}

opt_status enqueue_solve(opt_problem* pb, const opt_solve_params& p, bool lm, cudaStream_t st) {
  const float dmin = (float)p.diag_min, dmax = (float)p.diag_max;
  CKS(copy_planes_in(pb, pb->x, pb->user_x, pb->nx, st));
  k_reset<<<1, 32, 0, st>>>(pb->d_s, 1, lm ? p.lambda0 : 0.0);
  const bool fused = use_fused(pb, p) && p.inner > 0;
  const bool coop = !fused && use_persistent(pb, p);
  if (coop) CK(cudaMemsetAsync(pb->d_gbar, 0, sizeof(GridBarrier), st));
  for (int k = 0; k < p.outer; ++k) {
    // from the second outer iteration on, cos / sin of theta come from the
    // previous outer update (wide warps)
    const int csn_next = k + 1 < p.outer;
    st_init(pb, st, k, dmin, dmax, k > 0);
    if (p.materialized) csr_evalj(pb, st, p.materialized);
    if (fused) {
      for (int i = 0; i < p.inner; ++i) launch_grid_fused(pb->kind, grid_launch(pb, st), i);
      // Gauss-Newton: the last step and x += delta in one pass
      launch_grid_fused_fin(pb->kind, grid_launch(pb, st), p.inner, lm ? 0 : 1, lm ? 0 : csn_next);
    } else if (coop) {
      // the barrier's counter restarts at 0 (a timed-out launch may leave it
      // mid-count); its timeout flag accumulates over the solve
      CK(cudaMemsetAsync(&pb->d_gbar->count, 0, sizeof(unsigned int), st));
      CK(launch_grid_pcg_coop(grid_launch(pb, st), pb->d_gbar, 0, p.inner));
    } else {
      for (int i = 0; i < p.inner; ++i) {
        if (p.materialized) csr_apply(pb, st, i, p.materialized);
        else st_apply(pb, st, nullptr, i, 1);
        st_update(pb, st, i);
      }
    }
    if (!lm) {
      if (!fused) st_step(pb, st, 0, csn_next);
    } else {
      st_energy(pb, st, 1, -2);
      k_lm_decide<<<1, 32, 0, st>>>(pb->d_s, 1, p.eta, p.lambda_min, p.lambda_max, p.rel_tol);
      st_step(pb, st, 1, csn_next);
    }
  }
  st_energy(pb, st, 0, lm ? -1 : p.outer);
  CKS(copy_planes_out(pb, pb->user_x, pb->x, pb->nx, st));
  CK(cudaGetLastError());
  return OPT_OK;
}

std::vector<double> graph_key(const opt_solve_params& p, bool lm, cudaStream_t) {
  return {double(p.outer), double(p.inner), double(lm), double(p.use_precond), p.lambda0, p.lambda_min,
          p.lambda_max, p.diag_min, p.diag_max, p.eta, p.rel_tol, double(p.materialized), double(p.persistent),
          double(p.pcg_form)};
}

opt_status ensure_ehist(opt_problem* pb, int n) {
  if (pb->Ehist_cap >= n) return OPT_OK;
  if (pb->gexec) {
    cudaGraphExecDestroy(pb->gexec);
    pb->gexec = nullptr;
    pb->gkey.clear();
  }
  double* e = nullptr;
  CKS(dalloc(pb, &e, (size_t)n));
  pb->d_Ehist = e;
  pb->Ehist_cap = n;
  return OPT_OK;
}

opt_status run_solve(opt_problem* pb, const opt_solve_params* prm_in, opt_report* rep, bool lm) {
  if (!pb) return OPT_ERR_INVALID_ARG;
  opt_solve_params p;
  if (prm_in) p = *prm_in;
  else opt_solve_params_default(&p);
  CKS(check_params(p, lm));
  if (p.materialized < 0 || p.materialized > 2) return OPT_ERR_INVALID_ARG;
  if (p.pcg_form < 0 || p.pcg_form > 1) return OPT_ERR_INVALID_ARG;
  if (p.materialized && (pb->kind == K_WARPG || pb->kind == K_EMBED)) return OPT_ERR_INVALID_ARG;   // no CSR form
  if (p.materialized) CKS(csr_build(pb, p.materialized));
  cudaStream_t st = (cudaStream_t)p.stream;
  CK(cudaStreamSynchronize(st));
  CKS(ensure_ehist(pb, p.outer + 1));
  set_flags(pb, lm ? 1 : 0, p.use_precond, pb->d_Ehist);
  CKS(upload_desc(pb, st));
  if (p.use_graph) {
    const std::vector<double> key = graph_key(p, lm, st);
    if (!pb->gexec || key != pb->gkey) {
      if (pb->gexec) {
        cudaGraphExecDestroy(pb->gexec);
        pb->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(pb->cap_stream, cudaStreamCaptureModeThreadLocal));
      opt_status s = enqueue_solve(pb, p, lm, pb->cap_stream);
      cudaError_t e = cudaStreamEndCapture(pb->cap_stream, &g);
      if (s != OPT_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&pb->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      pb->gkey = key;
    }
    CK(cudaEventRecord(pb->ev0, st));
    CK(cudaGraphLaunch(pb->gexec, st));
    CK(cudaEventRecord(pb->ev1, st));
  } else {
    CK(cudaEventRecord(pb->ev0, st));
    CKS(enqueue_solve(pb, p, lm, st));
    CK(cudaEventRecord(pb->ev1, st));
  }
  CK(cudaEventSynchronize(pb->ev1));
  Scalars s;
  CK(cudaMemcpy(&s, pb->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  const int outer_done = lm ? s.outer_done : p.outer;
  std::vector<double> eh;
  CKS(download(eh, pb->d_Ehist, (size_t)outer_done + 1));
  pb->pcg_par = 0;
  if (rep) {
    rep->outer_done = outer_done;
    rep->pcg_done = s.pcg_iters;
    rep->accepted = lm ? s.accepted_total : p.outer;
    rep->converged = s.converged;
    rep->E0 = eh[0];
    rep->E_final = eh[outer_done];
    rep->lambda_final = lm ? s.lambda : 0.0;
    if (rep->E_history) std::memcpy(rep->E_history, eh.data(), eh.size() * sizeof(double));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pb->ev0, pb->ev1));
    rep->ms = ms;
  }
  if (use_persistent(pb, p)) {
    GridBarrier gb;
    CK(cudaMemcpy(&gb, pb->d_gbar, sizeof(gb), cudaMemcpyDeviceToHost));
    if (gb.timeout) return OPT_ERR_TIMEOUT;
  }
  if (s.timeout) return OPT_ERR_TIMEOUT;
  if (s.misaligned) return OPT_ERR_CUDA;
  if (s.nonfinite) return OPT_ERR_NUMERIC;
  return OPT_OK;
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link-time dependency on the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor maps of a grid with 128-pixel tiles (GridProb::tmap): [0] the nfp
// float planes of the slab, [1] the nx unknown planes, [2] the byte plane
// (if any).  Boxes: WIDE_BOX_W x HH x 1 floats, WIDE_BYTE_BOX_W x HH bytes;
// out-of-range elements are zero-filled.  All bases are device allocations
// (256-byte aligned) and every stride (P * 4, plane * 4, P) is a multiple of
// 16 bytes because P is a multiple of 128.
static opt_status make_grid_tmaps(opt_problem* q, const float* slab, int nfp, const uint8_t* bytes) {
  // L2 fill granularity of the copies (measured at 4096^2: 256-byte fills
  // suit the warp, whose neighbouring tiles reuse them, 64-byte fills the
  // Poisson kernels, 2-4 % apart)
  const CUtensorMapL2promotion l2 =
      q->kind == K_WARP ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cuda_fail(cudaErrorNotSupported, "cuTensorMapEncodeTiled");
  CUtensorMap maps[3];
  std::memset(maps, 0, sizeof(maps));
  const cuuint64_t P = (cuuint64_t)q->P, H = (cuuint64_t)q->H, pl = (cuuint64_t)q->plane;
  const cuuint32_t es[3] = {1, 1, 1};
  const cuuint32_t box3[3] = {(cuuint32_t)WIDE_BOX_W, (cuuint32_t)HH, 1};
  const cuuint64_t str3[2] = {P * 4, pl * 4};
  auto f32 = [&](CUtensorMap* m, const float* base, int planes) {
    const cuuint64_t dims[3] = {P, H, (cuuint64_t)planes};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, str3, box3, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  };
  if (f32(&maps[0], slab, nfp) != CUDA_SUCCESS || f32(&maps[1], q->x, q->nx) != CUDA_SUCCESS)
    return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
  if (bytes) {
    const cuuint64_t dims[2] = {P, H}, str[1] = {P};
    const cuuint32_t box[2] = {(cuuint32_t)WIDE_BYTE_BOX_W, (cuuint32_t)HH};
    if (enc(&maps[2], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(bytes), dims, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
  }
  static_assert(sizeof(CUtensorMap) == 128, "tensor maps are 128 bytes");
  unsigned long long* dmap = nullptr;
  CKS(dalloc(q, &dmap, 3 * sizeof(CUtensorMap) / sizeof(unsigned long long)));
  CK(cudaMemcpy(dmap, maps, sizeof(maps), cudaMemcpyHostToDevice));
  q->hg.tmap = dmap;
  return OPT_OK;
}

// Builds chunks of `per` consecutive units (tiles, vertex tiles or edges).
std::vector<Chunk> make_chunks(int n_units, int per, int prob) {
  std::vector<Chunk> ch;
  for (int b = 0; b < std::max(n_units, 1); b += per) ch.push_back(Chunk{prob, b, std::min(b + per, n_units), 0});
  return ch;
}

// Splits n_units into exactly min(n_units, n_chunks) chunks whose sizes differ
// by at most one unit (grids sized to a multiple of the SM count).  The larger
// chunks come first: blocks are dispatched in index order, so with two blocks
// per SM the first wave takes the larger chunks and no SM holds two of them
// (1024^2 warp, 1024 tiles on 304 blocks: at most 7 tiles per SM instead of 8;
// measured 7 % less time per solve than spreading the larger chunks evenly).
std::vector<Chunk> make_chunks_balanced(int n_units, int n_chunks, int prob) {
  std::vector<Chunk> ch;
  const int n = std::max(n_units, 1);
  const int c = std::max(1, std::min(n, n_chunks));
  const int q = n / c, rem = n % c;
  for (int k = 0; k < c; ++k) {
    const int b = k * q + std::min(k, rem);
    ch.push_back(Chunk{prob, b, std::min(b + q + (k < rem ? 1 : 0), n_units), 0});
  }
  return ch;
}

// Default work split: two blocks per SM (the residency of the wide-tile
// kernels), balanced.
constexpr int kDefaultBlocksPerSM = 2;

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

opt_status opt_solve_params_default(opt_solve_params* p) {
  if (!p) return OPT_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->outer = 10;
  p->inner = 10;
  p->lambda0 = 1e-3;
  p->lambda_min = 1e-16;
  p->lambda_max = 1e32;
  p->diag_min = 1e-6;
  p->diag_max = 1e32;
  p->eta = 1e-3;
  p->rel_tol = 0.0;
  p->use_precond = 1;
  p->materialized = 0;
  p->use_graph = 1;
  p->persistent = 0;
  p->stream = nullptr;
  return OPT_OK;
}

opt_status opt_selftest_grid_barrier(int32_t extra, int32_t rounds, int32_t* timed_out) {
  if (!timed_out || extra < 0 || extra > 64 || rounds < 1 || rounds > 1000) return OPT_ERR_INVALID_ARG;
  GridBarrier* gb = nullptr;
  CK(cudaMalloc(&gb, sizeof(GridBarrier)));
  GridBarrier h{};
  cudaError_t e = cudaMemset(gb, 0, sizeof(GridBarrier));
  if (e == cudaSuccess) e = launch_barrier_selftest(gb, 2, 2u + (unsigned)extra, rounds, 50000000ull, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, gb, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(gb);
  if (e != cudaSuccess) return cuda_fail(e, "opt_selftest_grid_barrier");
  *timed_out = h.timeout ? 1 : 0;
  return OPT_OK;
}

opt_status opt_selftest_staging_wait(int32_t complete, int32_t* timed_out) {
  if (!timed_out || complete < 0 || complete > 1) return OPT_ERR_INVALID_ARG;
  int* d = nullptr;
  CK(cudaMalloc(&d, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) e = launch_staging_selftest(complete, 50000000ull, d, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "opt_selftest_staging_wait");
  *timed_out = h ? 1 : 0;
  return OPT_OK;
}

const char* opt_status_str(opt_status s) {
  switch (s) {
    case OPT_OK: return "OPT_OK";
    case OPT_ERR_INVALID_ARG: return "OPT_ERR_INVALID_ARG";
    case OPT_ERR_OOM: return "OPT_ERR_OOM";
    case OPT_ERR_CUDA: return "OPT_ERR_CUDA";
    case OPT_ERR_NUMERIC: return "OPT_ERR_NUMERIC";
    case OPT_ERR_TIMEOUT: return "OPT_ERR_TIMEOUT";
    case OPT_ERR_BUDGET: return "OPT_ERR_BUDGET";
    case OPT_ERR_NOT_READY: return "OPT_ERR_NOT_READY";
  }
  return "OPT_ERR_UNKNOWN";
}

const char* opt_last_error(void) { return g_err.c_str(); }

opt_status opt_problem_create_grid(const opt_grid_desc* d, const opt_solve_params* prm, opt_problem** out) {
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d) return OPT_ERR_INVALID_ARG;
  if (d->kind != OPT_ARAP_WARP_2D && d->kind != OPT_POISSON_2D) return OPT_ERR_INVALID_ARG;
  if (d->W < 1 || d->H < 1 || d->W >= 32768 || d->H >= 32768) return OPT_ERR_INVALID_ARG;
  const bool warp = d->kind == OPT_ARAP_WARP_2D;
  const int nx = warp ? 3 : 4, nc = warp ? 2 : 4, nm = warp ? 2 : 1;
  // tile width: 128-pixel tiles (float4 rows) for grids at least 128 wide
  // (measured: 3 % faster for the batch of 512 uneven warps than from 256 up),
  // 32-pixel tiles otherwise
  const int req_tw = prm ? prm->tile_w : 0;
  if (req_tw != 0 && req_tw != 32 && req_tw != 128) return OPT_ERR_INVALID_ARG;
  const int tw = req_tw ? req_tw : (d->W >= 128 ? 128 : 32);
  for (int c = 0; c < nx; ++c)
    if (!d->unknowns[c]) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < nc; ++c)
    if (!d->consts[c]) return OPT_ERR_INVALID_ARG;
  const int nh = warp ? d->n_handles : 0;
  if (nh < 0) return OPT_ERR_INVALID_ARG;
  if (nh > 0 && (!d->handle_idx || !d->handle_target)) return OPT_ERR_INVALID_ARG;
  if (warp && (!std::isfinite(d->w_reg) || !std::isfinite(d->w_fit) || d->w_reg < 0.f || d->w_fit < 0.f))
    return OPT_ERR_INVALID_ARG;

  if (tw == 128) CK(grid_kernels_prepare());
  std::unique_ptr<opt_problem> pb(new opt_problem());
  pb->kind = warp ? K_WARP : K_POISSON;
  pb->tile_w = tw;
  pb->grid_desc = *d;
  pb->has_grid_desc = true;
  pb->nx = nx;
  pb->nm = nm;
  pb->W = d->W;
  pb->H = d->H;
  pb->P = round_up(d->W, tw);
  pb->plane = (long long)pb->P * d->H;
  pb->ulen = (long long)d->W * d->H;
  CKS(common_setup(pb.get()));
  const int W = d->W, H = d->H, P = pb->P;
  const size_t n = (size_t)W * H;

  // host copies of the constants for validation and planning
  std::vector<float> cst;
  for (int c = 0; c < nc; ++c) {
    std::vector<float> tmp;
    CKS(download(tmp, d->consts[c], n));
    if (!all_finite(tmp)) return OPT_ERR_INVALID_ARG;
  }
  std::vector<uint8_t> mask;
  if (d->mask) CKS(download(mask, d->mask, n));
  std::vector<int> hidx;
  std::vector<float> htgt;
  if (nh > 0) {
    CKS(download(hidx, d->handle_idx, (size_t)nh));
    CKS(download(htgt, d->handle_target, (size_t)nh * 2));
    if (!all_finite(htgt)) return OPT_ERR_INVALID_ARG;
    std::vector<int> sorted(hidx);
    std::sort(sorted.begin(), sorted.end());
    for (size_t i = 0; i < sorted.size(); ++i) {
      if (sorted[i] < 0 || (size_t)sorted[i] >= n) return OPT_ERR_INVALID_ARG;
      if (i && sorted[i] == sorted[i - 1]) return OPT_ERR_INVALID_ARG;
    }
  }

  // active tiles: at least one unmasked (warp) / free (Poisson) pixel
  const int ntx = (W + tw - 1) / tw, nty = (H + TH - 1) / TH;
  std::vector<int> tiles;
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx) {
      bool act = mask.empty();
      for (int y = ty * TH; !act && y < std::min(H, ty * TH + TH); ++y)
        for (int x = tx * tw; x < std::min(W, tx * tw + tw); ++x)
          if (mask[(size_t)y * W + x] == 0) { act = true; break; }
      if (act) tiles.push_back((ty << 16) | tx);
    }
  if (tiles.empty()) tiles.push_back(0);
  std::vector<Chunk> chunks = make_chunks_balanced((int)tiles.size(), pb->sms * kDefaultBlocksPerSM, 0);

  // handles sorted by tile
  std::vector<int> order(nh);
  std::iota(order.begin(), order.end(), 0);
  auto tile_of = [&](int pix) { return (pix / W / TH) * ntx + (pix % W) / tw; };
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const int ta = tile_of(hidx[a]), tb = tile_of(hidx[b]);
    return ta != tb ? ta < tb : hidx[a] < hidx[b];
  });
  std::vector<int> hbeg((size_t)ntx * nty + 1, 0), hpix(nh);
  std::vector<float> hts((size_t)nh * 2);
  for (int k = 0; k < nh; ++k) {
    const int i = order[k], pix = hidx[i];
    hpix[k] = (pix / W) * P + (pix % W);
    hts[2 * k] = htgt[2 * i];
    hts[2 * k + 1] = htgt[2 * i + 1];
    hbeg[tile_of(pix) + 1] += 1;
  }
  for (size_t t = 1; t < hbeg.size(); ++t) hbeg[t] += hbeg[t - 1];

  // device buffers
  opt_problem* q = pb.get();
  const size_t pl = (size_t)pb->plane;
  float *c = nullptr, *m = nullptr, *dc = nullptr;
  uint8_t* dmask = nullptr;
  int *dhbeg = nullptr, *dhpix = nullptr;
  float* dhtgt = nullptr;
  CKS(dalloc(q, &q->x, nx * pl));
  CKS(dalloc(q, &dc, nm * pl));
  // one slab for every plane the PCG launches touch, in the order r, M^-1,
  // p (two), q, delta, cos / sin, constants, mask, degree bytes (planes are
  // multiples of 32 floats, so every plane stays 128-byte aligned)
  const bool has_csn = warp && tw == 128;
  const bool has_sdeg = !warp && tw == 128;
  // 128-pixel tiles: the single-reduction PCG's double-buffered z and w planes
  const int nzw = tw == 128 ? 4 * nx : 0;
  const int nfp = nx + nm + 2 * nx + nx + nx + (has_csn ? 2 : 0) + nc + nzw;
  const size_t nslab = (size_t)nfp * pl + (d->mask ? pl / 4 : 0) + (has_sdeg ? pl / 4 : 0);
  float* slab = nullptr;
  CKS(dalloc(q, &slab, nslab));
  float* cur = slab;
  auto take = [&](size_t n) { float* r = cur; cur += n; return r; };
  q->rvec = take(nx * pl);
  m = take(nm * pl);
  q->pbuf = take(2 * nx * pl);
  q->qvec = take(nx * pl);
  q->dvec = take(nx * pl);
  float* csn = has_csn ? take(2 * pl) : nullptr;
  c = take(nc * pl);
  float* zb = nzw ? take(2 * nx * pl) : nullptr;
  float* wb = nzw ? take(2 * nx * pl) : nullptr;
  if (d->mask) dmask = reinterpret_cast<uint8_t*>(take(pl / 4));
  uint8_t* dsdeg = has_sdeg ? reinterpret_cast<uint8_t*>(take(pl / 4)) : nullptr;
  if (has_csn) {
    CKS(dalloc(q, &q->d_gbar, 1));
    q->coop_cap = grid_coop_capacity(d->mask != nullptr);
  }
  if (d->mask) CK(cudaMemcpy2D(dmask, P, d->mask, W, W, H, cudaMemcpyDeviceToDevice));
  if (has_sdeg) {
    launch_pois_sdeg(W, H, P, dmask, dsdeg, nullptr);
    CK(cudaGetLastError());
  }
  // Poisson, 128-pixel tiles with fixed pixels: the quads holding a free
  // pixel (one word per row and tile column, bit l for the quad at
  // 128 tx + 4 l); the vector update skips the others
  unsigned int* dlive = nullptr;
  if (has_sdeg && !mask.empty()) {
    std::vector<unsigned int> lv((size_t)H * ntx, 0u);
    for (int y = 0; y < H; ++y) {
      const uint8_t* mr = mask.data() + (size_t)y * W;
      for (int x = 0; x < W; ++x)
        if (mr[x] == 0) lv[(size_t)y * ntx + x / 128] |= 1u << ((x % 128) / 4);
    }
    CKS(dalloc(q, &dlive, lv.size()));
    CKS(upload(dlive, lv));
  }
  for (int k = 0; k < nc; ++k)
    CK(cudaMemcpy2D(c + k * pl, (size_t)P * 4, d->consts[k], (size_t)W * 4, (size_t)W * 4, H,
                    cudaMemcpyDeviceToDevice));
  CKS(dalloc(q, &dhbeg, hbeg.size()));
  CKS(upload(dhbeg, hbeg));
  CKS(dalloc(q, &dhpix, hpix.size()));
  CKS(upload(dhpix, hpix));
  CKS(dalloc(q, &dhtgt, hts.size()));
  CKS(upload(dhtgt, hts));
  CKS(dalloc(q, &q->d_tiles, tiles.size()));
  CKS(upload(q->d_tiles, tiles));
  q->h_tiles = tiles;
  q->ntiles = (int)tiles.size();
  CKS(dalloc(q, &q->d_chunks, chunks.size()));
  CKS(upload(q->d_chunks, chunks));
  q->h_chunks = chunks;
  q->nchunks = (int)chunks.size();
  CKS(dalloc(q, &q->d_part, 4 * chunks.size()));   // up to three partials per chunk
  CKS(dalloc(q, &q->dg, 1));
  for (int k = 0; k < nx; ++k) q->user_x[k] = d->unknowns[k];
  q->h_mask = mask;
  q->h_hpix = hpix;

  GridProb& g = q->hg;
  g.kind = q->kind;
  g.W = W; g.H = H; g.P = P;
  g.tw = tw;
  g.csn = csn;
  g.ntx = ntx; g.nty = nty;
  g.plane = (long long)pl;
  g.chunk_begin = 0;
  g.chunk_end = q->nchunks;
  g.w_reg = warp ? d->w_reg : 1.f;
  g.w_fit = warp ? d->w_fit : 0.f;
  g.s_w = std::sqrt(g.w_reg);
  g.s_f = std::sqrt(g.w_fit);
  g.use_precond = 1;
  g.lm = 0;
  g.x = q->x; g.c = c; g.mask = dmask; g.sdeg = dsdeg;
  g.live = dlive;
  // 128-pixel tiles: tensor maps of the staged planes, and where each plane
  // group lies in the slab
  g.tmap = nullptr;
  const auto zof = [&](const float* ptr) { return ptr ? (int)((ptr - slab) / (ptrdiff_t)pl) : -1; };
  g.zpack = zof(q->rvec) | zof(m) << 6 | zof(q->pbuf) << 12 | (csn ? zof(csn) : 0) << 18 | zof(c) << 24;
  g.zb = zb;
  g.wb = wb;
  g.zpack2 = zb ? (zof(zb) | zof(wb) << 6) : 0;
  if (tw == 128) CKS(make_grid_tmaps(q, slab, nfp, warp ? dmask : dsdeg));
  g.d = q->dvec; g.r = q->rvec; g.p = q->pbuf; g.q = q->qvec; g.m = m; g.dc = dc;
  g.hbeg = dhbeg; g.hpix = dhpix; g.htgt = dhtgt;
  g.jtf_out = nullptr; g.diag_out = nullptr;
  g.s = q->d_s;
  g.Ehist = nullptr;
  CKS(upload_desc(q, nullptr));
  *out = pb.release();
  return OPT_OK;
}

// Graph planning for dimension D: D = 3 is the ARAP mesh (unknowns dx, dy, dz,
// ax, ay, az; rest positions and targets in 3-D), D = 2 the warp on a graph
// (unknowns dx, dy, theta; rest positions and targets in 2-D).
// grid3 (volumetric problems): the W x H x D voxel grid whose 7-point stencil
// the host edge lists hold; vertices then keep the caller's order (already
// local) and the gather kernels take neighbours from the stencil.
// Embedded deformation: the 12 unknown planes and the constraint weight
// (the rest of the problem is an opt_graph_desc).
struct EmbedExtra {
  float* unknowns[12];
  float w_rot;
};

static opt_status create_graph_impl(const opt_graph_desc* d, int D, opt_problem** out,
                                    const std::vector<int>* host_e0 = nullptr,
                                    const std::vector<int>* host_e1 = nullptr, const int* grid3 = nullptr,
                                    const EmbedExtra* ed = nullptr) {
  // unknown planes, distinct-diagonal planes, geometry and vector records per vertex
  const int NXg = ed ? 12 : (D == 3 ? 6 : 3), NMg = ed ? 10 : (D == 3 ? 4 : 2);
  const int NGR = ed ? 1 : (D == 3 ? 3 : 1), NVR = ed ? 3 : (D == 3 ? 2 : 1);
  float* const* ux = ed ? ed->unknowns : d ? d->unknowns : nullptr;
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d) return OPT_ERR_INVALID_ARG;
  if (d->V < 1 || d->E < 0 || d->n_handles < 0) return OPT_ERR_INVALID_ARG;
  if (d->E > 0 && !host_e0 && (!d->v0 || !d->v1)) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < NXg; ++c)
    if (!ux[c]) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < D; ++c)
    if (!d->urshape[c]) return OPT_ERR_INVALID_ARG;
  if (ed && (!std::isfinite(ed->w_rot) || ed->w_rot < 0.f)) return OPT_ERR_INVALID_ARG;
  if (d->n_handles > 0 && (!d->handle_idx || !d->handle_target)) return OPT_ERR_INVALID_ARG;
  if (!std::isfinite(d->w_reg) || !std::isfinite(d->w_fit) || d->w_reg < 0.f || d->w_fit < 0.f)
    return OPT_ERR_INVALID_ARG;

  std::unique_ptr<opt_problem> pb(new opt_problem());
  opt_problem* q = pb.get();
  q->kind = ed ? K_EMBED : (grid3 ? K_VOLUME : (D == 3 ? K_MESH : K_WARPG));
  q->nx = NXg;
  q->nm = NMg;
  q->V = d->V;
  q->E = d->E;
  const int V = d->V, E = d->E, nh = d->n_handles;
  const int Vp = round_up(V, 32);
  q->plane = Vp;
  q->ulen = V;
  CKS(common_setup(q));

  std::vector<int> e0, e1;
  if (host_e0) {
    e0 = *host_e0;
    e1 = *host_e1;
  } else {
    CKS(download(e0, d->v0, (size_t)E));
    CKS(download(e1, d->v1, (size_t)E));
  }
  for (int e = 0; e < E; ++e)
    if (e0[e] < 0 || e0[e] >= V || e1[e] < 0 || e1[e] >= V || e0[e] == e1[e]) return OPT_ERR_INVALID_ARG;
  std::vector<float> Uh[3];
  Uh[2].assign((size_t)V, 0.f);             // a graph warp lies in the plane z = 0
  for (int c = 0; c < D; ++c) {
    CKS(download(Uh[c], d->urshape[c], (size_t)V));
    if (!all_finite(Uh[c])) return OPT_ERR_INVALID_ARG;
  }
  // internal vertex order: internal k = caller perm[k]; edges and handles are
  // renumbered before sorting
  std::vector<int> perm;
  if (grid3) {
    perm.resize((size_t)V);
    std::iota(perm.begin(), perm.end(), 0);
  } else {
    perm = morton_order(Uh, V);
  }
  std::vector<int> iperm((size_t)V);
  for (int k = 0; k < V; ++k) iperm[perm[k]] = k;
  for (int e = 0; e < E; ++e) { e0[e] = iperm[e0[e]]; e1[e] = iperm[e1[e]]; }
  bool sorted = true;
  for (int e = 1; e < E && sorted; ++e)
    if (e0[e] < e0[e - 1] || (e0[e] == e0[e - 1] && e1[e] < e1[e - 1])) sorted = false;
  if (!sorted) {
    // counting sort by v0, then each (short) row by v1
    std::vector<int> start((size_t)V + 1, 0), s1((size_t)E);
    for (int e = 0; e < E; ++e) start[(size_t)e0[e] + 1] += 1;
    for (int v = 0; v < V; ++v) start[(size_t)v + 1] += start[v];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int e = 0; e < E; ++e) s1[(size_t)fill[e0[e]]++] = e1[e];
    for (int v = 0; v < V; ++v) {
      const int b = start[v], e = start[(size_t)v + 1];
      for (int k = b + 1; k < e; ++k) {   // rows are short: insertion sort
        const int x = s1[k];
        int m = k;
        for (; m > b && s1[(size_t)m - 1] > x; --m) s1[m] = s1[(size_t)m - 1];
        s1[m] = x;
      }
      for (int k = b; k < e; ++k) e0[k] = v;
    }
    e1.swap(s1);
  }
  std::vector<int> hidx;
  std::vector<float> htgt;
  if (nh > 0) {
    CKS(download(hidx, d->handle_idx, (size_t)nh));
    CKS(download(htgt, d->handle_target, (size_t)nh * D));
    if (!all_finite(htgt)) return OPT_ERR_INVALID_ARG;
    for (int& h : hidx) {
      if (h < 0 || h >= V) return OPT_ERR_INVALID_ARG;
      h = iperm[h];
    }
  }
  std::vector<int> order(nh);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return hidx[a] < hidx[b]; });
  const int nvt = (V + VT - 1) / VT;
  std::vector<int> hbeg((size_t)nvt + 1, 0), hpix(nh);
  std::vector<float> hts((size_t)nh * D);
  std::vector<float> degw((size_t)V, 0.f);
  for (int k = 0; k < nh; ++k) {
    const int i = order[k], v = hidx[i];
    if (v < 0 || v >= V || (k && hpix[k - 1] == v)) return OPT_ERR_INVALID_ARG;
    hpix[k] = v;
    for (int c = 0; c < D; ++c) hts[(size_t)D * k + c] = htgt[(size_t)D * i + c];
    hbeg[v / VT + 1] += 1;
    degw[v] += d->w_fit;
  }
  for (size_t t = 1; t < hbeg.size(); ++t) hbeg[t] += hbeg[t - 1];
  for (int e = 0; e < E; ++e) {
    degw[e0[e]] += d->w_reg;
    degw[e1[e]] += d->w_reg;
  }
  // out-edge rows of the sorted list, and the in-edges of every vertex
  // (sources ascending, as the sorted list visits them)
  std::vector<int> orow((size_t)V + 1, 0), irow((size_t)V + 1, 0), isrc((size_t)E);
  for (int e = 0; e < E; ++e) {
    orow[(size_t)e0[e] + 1] += 1;
    irow[(size_t)e1[e] + 1] += 1;
  }
  for (int v = 0; v < V; ++v) {
    orow[(size_t)v + 1] += orow[v];
    irow[(size_t)v + 1] += irow[v];
  }
  {
    std::vector<int> fill(irow.begin(), irow.end() - 1);
    for (int e = 0; e < E; ++e) isrc[(size_t)fill[e1[e]]++] = e0[e];
  }

  const int target = std::max(1, q->sms * 8);
  std::vector<Chunk> vch = make_chunks_balanced(nvt, target, 0);
  for (Chunk& c : vch) { c.begin *= VT; c.end = std::min(V, c.end * VT); }
  std::vector<Chunk> ech = make_chunks_balanced(E, target, 0);

  const size_t pl = (size_t)Vp;
  float *U = nullptr, *dgw = nullptr, *m = nullptr, *dc = nullptr, *dhtgt = nullptr;
  int *de0 = nullptr, *de1 = nullptr, *dhbeg = nullptr, *dhpix = nullptr;
  CKS(dalloc(q, &q->x, NXg * pl));
  CKS(dalloc(q, &U, D * pl));
  CKS(dalloc(q, &dgw, pl));
  CKS(dalloc(q, &q->dvec, NXg * pl));
  CKS(dalloc(q, &q->rvec, NXg * pl));
  CKS(dalloc(q, &q->qvec, NXg * pl));
  CKS(dalloc(q, &q->pbuf, 2 * NXg * pl));
  CKS(dalloc(q, &m, NMg * pl));
  CKS(dalloc(q, &dc, NMg * pl));
  float4 *grec = nullptr, *vrec = nullptr;
  CKS(dalloc(q, &grec, (size_t)NGR * V));
  CKS(dalloc(q, &vrec, (size_t)NVR * V));
  int *dorow = nullptr, *dirow = nullptr, *disrc = nullptr;
  CKS(dalloc(q, &dorow, orow.size()));
  CKS(upload(dorow, orow));
  CKS(dalloc(q, &dirow, irow.size()));
  CKS(upload(dirow, irow));
  CKS(dalloc(q, &disrc, std::max<size_t>(1, isrc.size())));
  if (E > 0) CKS(upload(disrc, isrc));
  for (int c = 0; c < D; ++c) {
    std::vector<float> Ui((size_t)V);
    for (int k = 0; k < V; ++k) Ui[k] = Uh[c][perm[k]];
    CKS(upload(U + c * pl, Ui));
  }
  CKS(dalloc(q, &q->d_perm, (size_t)V));
  CKS(upload(q->d_perm, perm));
  CKS(upload(dgw, degw));
  CKS(dalloc(q, &de0, (size_t)E));
  CKS(upload(de0, e0));
  CKS(dalloc(q, &de1, (size_t)E));
  CKS(upload(de1, e1));
  CKS(dalloc(q, &dhbeg, hbeg.size()));
  CKS(upload(dhbeg, hbeg));
  CKS(dalloc(q, &dhpix, hpix.size()));
  CKS(upload(dhpix, hpix));
  CKS(dalloc(q, &dhtgt, hts.size()));
  CKS(upload(dhtgt, hts));
  CKS(dalloc(q, &q->d_vchunks, vch.size()));
  CKS(upload(q->d_vchunks, vch));
  CKS(dalloc(q, &q->d_echunks, ech.size()));
  CKS(upload(q->d_echunks, ech));
  q->h_vch = vch;
  q->h_ech = ech;
  q->tileable = !ed && !grid3 && D == 3;
  q->nvchunks = (int)vch.size();
  q->nechunks = (int)ech.size();
  CKS(dalloc(q, &q->d_part, 2 * std::max(vch.size(), ech.size())));
  CKS(dalloc(q, &q->dm, 1));
  for (int k = 0; k < NXg; ++k) q->user_x[k] = ux[k];
  q->h_e0 = e0;
  q->h_e1 = e1;
  q->h_hpix = hpix;

  MeshProb& g = q->hm;
  g.V = V; g.E = E; g.Vp = Vp;
  g.vchunk_begin = 0; g.vchunk_end = q->nvchunks;
  g.echunk_begin = 0; g.echunk_end = q->nechunks;
  g.tchunk_begin = 0; g.tchunk_end = q->ntchunks;
  g.w_reg = d->w_reg; g.w_fit = d->w_fit;
  g.s_w = std::sqrt(d->w_reg); g.s_f = std::sqrt(d->w_fit);
  g.w_rot = ed ? ed->w_rot : 0.f; g.s_r = std::sqrt(g.w_rot);
  g.use_precond = 1; g.lm = 0;
  g.x = q->x; g.U = U; g.degw = dgw; g.e0 = de0; g.e1 = de1;
  g.d = q->dvec; g.r = q->rvec; g.p = q->pbuf; g.q = q->qvec; g.m = m; g.dc = dc;
  g.orow = dorow; g.irow = dirow; g.isrc = disrc;
  g.hptr = nullptr; g.hvtx = nullptr; g.lnbr = nullptr; g.rptr = nullptr; g.rin = nullptr; g.itslot = nullptr;
  g.gw = grid3 ? grid3[0] : 0; g.gh = grid3 ? grid3[1] : 0; g.gd = grid3 ? grid3[2] : 0; g.gpad = 0;
  g.grec = grec; g.vrec = vrec;
  g.hbeg = dhbeg; g.hpix = dhpix; g.htgt = dhtgt;
  g.jtf_out = nullptr; g.diag_out = nullptr;
  g.s = q->d_s;
  g.Ehist = nullptr;
  CKS(upload_desc(q, nullptr));
  *out = pb.release();
  return OPT_OK;
}

opt_status opt_problem_create_graph(const opt_graph_desc* d, const opt_solve_params* prm, opt_problem** out) {
  (void)prm;
  return create_graph_impl(d, 3, out);
}

opt_status opt_problem_create_graph2d(const opt_graph_desc* d, const opt_solve_params* prm, opt_problem** out) {
  (void)prm;
  return create_graph_impl(d, 2, out);
}

opt_status opt_problem_create_embedded(const opt_embedded_desc* d, const opt_solve_params* prm, opt_problem** out) {
  (void)prm;
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d) return OPT_ERR_INVALID_ARG;
  opt_graph_desc g = {};
  g.V = d->V;
  g.E = d->E;
  g.v0 = d->v0;
  g.v1 = d->v1;
  for (int c = 0; c < 3; ++c) g.urshape[c] = d->urshape[c];
  g.handle_idx = d->handle_idx;
  g.handle_target = d->handle_target;
  g.n_handles = d->n_handles;
  g.w_reg = d->w_reg;
  g.w_fit = d->w_fit;
  EmbedExtra ex;
  for (int c = 0; c < 12; ++c) ex.unknowns[c] = d->unknowns[c];
  ex.w_rot = d->w_rot;
  return create_graph_impl(&g, 3, out, nullptr, nullptr, nullptr, &ex);
}

opt_status opt_problem_create_volume(const opt_volume_desc* d, const opt_solve_params* prm, opt_problem** out) {
  (void)prm;
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d || d->W < 1 || d->H < 1 || d->D < 1) return OPT_ERR_INVALID_ARG;
  const long long V = (long long)d->W * d->H * d->D;
  if (V > (1ll << 27)) return OPT_ERR_INVALID_ARG;
  const int W = d->W, H = d->H, Dz = d->D;
  // the 7-point stencil as directed edges, sorted by (v0, v1)
  std::vector<int> e0, e1;
  e0.reserve((size_t)V * 6);
  e1.reserve((size_t)V * 6);
  for (int z = 0; z < Dz; ++z)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        const int i = (z * H + y) * W + x;
        const int WH = W * H;
        if (z > 0) { e0.push_back(i); e1.push_back(i - WH); }
        if (y > 0) { e0.push_back(i); e1.push_back(i - W); }
        if (x > 0) { e0.push_back(i); e1.push_back(i - 1); }
        if (x + 1 < W) { e0.push_back(i); e1.push_back(i + 1); }
        if (y + 1 < H) { e0.push_back(i); e1.push_back(i + W); }
        if (z + 1 < Dz) { e0.push_back(i); e1.push_back(i + WH); }
      }
  opt_graph_desc g = {};
  g.V = (int32_t)V;
  g.E = (int32_t)e0.size();
  for (int c = 0; c < 6; ++c) g.unknowns[c] = d->unknowns[c];
  for (int c = 0; c < 3; ++c) g.urshape[c] = d->urshape[c];
  g.handle_idx = d->handle_idx;
  g.handle_target = d->handle_target;
  g.n_handles = d->n_handles;
  g.w_reg = d->w_reg;
  g.w_fit = d->w_fit;
  const int dims[3] = {W, H, Dz};
  return create_graph_impl(&g, 3, out, &e0, &e1, dims);
}

opt_status opt_problem_destroy(opt_problem* prob) {
  if (!prob) return OPT_OK;
  cudaDeviceSynchronize();
  delete prob;
  return OPT_OK;
}

opt_status opt_solve_gn(opt_problem* prob, const opt_solve_params* params, opt_report* report) {
  return run_solve(prob, params, report, false);
}

opt_status opt_solve_lm(opt_problem* prob, const opt_solve_params* params, opt_report* report) {
  return run_solve(prob, params, report, true);
}

opt_status opt_problem_info(const opt_problem* prob, int64_t* n_unknowns, int32_t* n_planes, int64_t* plane_len) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  if (n_unknowns) *n_unknowns = (int64_t)prob->nx * prob->ulen;
  if (n_planes) *n_planes = prob->nx;
  if (plane_len) *plane_len = prob->ulen;
  return OPT_OK;
}

// --- parity hooks and step-wise PCG ------------------------------------------
static opt_status hook_prepare(opt_problem* pb, double lambda, bool with_outputs) {
  if (!pb->d_tmp) CKS(dalloc(pb, &pb->d_tmp, (size_t)pb->nx * pb->plane));
  if (with_outputs && !pb->d_jtf) {
    CKS(dalloc(pb, &pb->d_jtf, (size_t)pb->nx * pb->plane));
    CKS(dalloc(pb, &pb->d_diag, (size_t)pb->nm * pb->plane));
  }
  CK(cudaDeviceSynchronize());
  set_flags(pb, lambda != 0.0 ? 1 : 0, 1, nullptr);
  if (is_grid(pb)) {
    pb->hg.jtf_out = with_outputs ? pb->d_jtf : nullptr;
    pb->hg.diag_out = with_outputs ? pb->d_diag : nullptr;
  } else {
    pb->hm.jtf_out = with_outputs ? pb->d_jtf : nullptr;
    pb->hm.diag_out = with_outputs ? pb->d_diag : nullptr;
  }
  CKS(upload_desc(pb, nullptr));
  return OPT_OK;
}

static opt_status hook_finish(opt_problem* pb) {
  if (is_grid(pb)) {
    pb->hg.jtf_out = nullptr;
    pb->hg.diag_out = nullptr;
  } else {
    pb->hm.jtf_out = nullptr;
    pb->hm.diag_out = nullptr;
  }
  CKS(upload_desc(pb, nullptr));
  return OPT_OK;
}

static opt_status hook_init(opt_problem* pb, double lambda) {
  CKS(copy_planes_in(pb, pb->x, pb->user_x, pb->nx, nullptr));
  k_reset<<<1, 32>>>(pb->d_s, 1, lambda);
  st_init(pb, nullptr, -1, 1e-6f, 1e32f);
  CK(cudaGetLastError());
  return OPT_OK;
}

opt_status opt_pcg_init(opt_problem* prob, double lambda, double* energy) {
  if (!prob || !(lambda >= 0.0) || !std::isfinite(lambda)) return OPT_ERR_INVALID_ARG;
  CKS(hook_prepare(prob, lambda, false));
  CKS(hook_init(prob, lambda));
  CK(cudaDeviceSynchronize());
  prob->pcg_par = 0;
  Scalars s;
  CK(cudaMemcpy(&s, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  if (energy) *energy = s.E;
  if (s.timeout) return OPT_ERR_TIMEOUT;
  if (s.misaligned) return OPT_ERR_CUDA;
  return s.nonfinite ? OPT_ERR_NUMERIC : OPT_OK;
}

opt_status opt_pcg_step(opt_problem* prob, int32_t n_iters) {
  if (!prob || n_iters < 0) return OPT_ERR_INVALID_ARG;
  for (int i = 0; i < n_iters; ++i) {
    st_apply(prob, nullptr, nullptr, prob->pcg_par, 1);
    st_update(prob, nullptr, prob->pcg_par);
    prob->pcg_par += 1;
  }
  CK(cudaGetLastError());
  return OPT_OK;
}

opt_status opt_pcg_get_state(opt_problem* prob, float* delta, float* r, float* p, int32_t* iters_done) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  float* planes[12];
  if (delta) {
    dense_planes(prob, delta, planes, prob->nx);
    CKS(copy_planes_out(prob, planes, prob->dvec, prob->nx, nullptr));
  }
  if (r) {
    dense_planes(prob, r, planes, prob->nx);
    CKS(copy_planes_out(prob, planes, prob->rvec, prob->nx, nullptr));
  }
  if (p) {
    dense_planes(prob, p, planes, prob->nx);
    if (prob->pcg_par == 0) {
      for (int c = 0; c < prob->nx; ++c) CK(cudaMemset(planes[c], 0, (size_t)prob->ulen * 4));
    } else {
      const float* src = prob->pbuf + (size_t)(prob->pcg_par & 1) * prob->nx * prob->plane;
      CKS(copy_planes_out(prob, planes, src, prob->nx, nullptr));
    }
  }
  CK(cudaDeviceSynchronize());
  if (iters_done) {
    Scalars s;
    CK(cudaMemcpy(&s, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
    *iters_done = s.pcg_iters;
  }
  return OPT_OK;
}

opt_status opt_apply_jtj(opt_problem* prob, const float* p, float* q, double lambda, double* pq) {
  if (!prob || !p || !q || !(lambda >= 0.0) || !std::isfinite(lambda)) return OPT_ERR_INVALID_ARG;
  CKS(hook_prepare(prob, lambda, false));
  CKS(hook_init(prob, lambda));
  float* planes[12];
  dense_planes(prob, p, planes, prob->nx);
  CKS(copy_planes_in(prob, prob->d_tmp, planes, prob->nx, nullptr));
  k_force_active<<<1, 32>>>(prob->d_s, 1);
  st_apply(prob, nullptr, prob->d_tmp, 0, 0);
  CK(cudaGetLastError());
  dense_planes(prob, q, planes, prob->nx);
  CKS(copy_planes_out(prob, planes, prob->qvec, prob->nx, nullptr));
  CK(cudaDeviceSynchronize());
  Scalars s;
  CK(cudaMemcpy(&s, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  if (pq) *pq = s.pq;
  prob->pcg_par = 0;
  return OPT_OK;
}

opt_status opt_eval_jtf(opt_problem* prob, float* jtf, float* diag, double* energy) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  CKS(hook_prepare(prob, 0.0, true));
  CKS(hook_init(prob, 0.0));
  float* planes[12];
  if (jtf) {
    dense_planes(prob, jtf, planes, prob->nx);
    CKS(copy_planes_out(prob, planes, prob->d_jtf, prob->nx, nullptr));
  }
  if (diag) {
    dense_planes(prob, diag, planes, prob->nx);
    for (int c = 0; c < prob->nx; ++c) {
      float* one[1] = {planes[c]};
      CKS(copy_planes_out(prob, one, prob->d_diag + (size_t)mplane_of(prob->kind, c) * prob->plane, 1, nullptr));
    }
  }
  CK(cudaDeviceSynchronize());
  Scalars s;
  CK(cudaMemcpy(&s, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  if (energy) *energy = s.E;
  prob->pcg_par = 0;
  return hook_finish(prob);
}

opt_status opt_profile_pcg(opt_problem* prob, int32_t n_iters, void* stream, float* ms) {
  if (!prob || n_iters < 1 || !ms) return OPT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CKS(hook_prepare(prob, 0.0, false));
  const int nev = 2 * (1 + 2 * n_iters);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  opt_status status = OPT_OK;
  for (int i = 0; i < nev && status == OPT_OK; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) status = OPT_ERR_CUDA;
  if (status == OPT_OK) {
    copy_planes_in(prob, prob->x, prob->user_x, prob->nx, st);
    k_reset<<<1, 32, 0, st>>>(prob->d_s, 1, 0.0);
    // wide warps: PCGInit as a solve runs it from the second outer iteration
    // on, reading cos / sin of theta written ahead of it (not timed)
    const int csn = wide_warp(prob);
    if (csn) launch_grid_csn(grid_launch(prob, st));
    cudaEventRecord(ev[0], st);
    st_init(prob, st, -1, 1e-6f, 1e32f, csn);
    cudaEventRecord(ev[1], st);
    for (int i = 0; i < n_iters; ++i) {
      cudaEventRecord(ev[2 + 4 * i], st);
      st_apply(prob, st, nullptr, i, 1);
      cudaEventRecord(ev[3 + 4 * i], st);
      cudaEventRecord(ev[4 + 4 * i], st);
      st_update(prob, st, i);
      cudaEventRecord(ev[5 + 4 * i], st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_fail(e, "opt_profile_pcg");
  }
  if (status == OPT_OK) {
    float t = 0.f, a = 0.f, u = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    for (int i = 0; i < n_iters; ++i) {
      float x = 0.f, y = 0.f;
      cudaEventElapsedTime(&x, ev[2 + 4 * i], ev[3 + 4 * i]);
      cudaEventElapsedTime(&y, ev[4 + 4 * i], ev[5 + 4 * i]);
      a += x;
      u += y;
    }
    ms[0] = t;
    ms[1] = a / n_iters;
    ms[2] = u / n_iters;
    prob->pcg_par = n_iters;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return status;
}

opt_status opt_profile_pcg_fused(opt_problem* prob, int32_t n_iters, void* stream, float* ms) {
  if (!prob || n_iters < 2 || !ms) return OPT_ERR_INVALID_ARG;
  if ((prob->kind != K_WARP && prob->kind != K_POISSON) || !prob->hg.zb) return OPT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CKS(hook_prepare(prob, 0.0, false));
  const int nev = 2 * (n_iters + 2);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  opt_status status = OPT_OK;
  for (int i = 0; i < nev && status == OPT_OK; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) status = OPT_ERR_CUDA;
  if (status == OPT_OK) {
    copy_planes_in(prob, prob->x, prob->user_x, prob->nx, st);
    k_reset<<<1, 32, 0, st>>>(prob->d_s, 1, 0.0);
    const int csn = wide_warp(prob);
    if (csn) launch_grid_csn(grid_launch(prob, st));
    cudaEventRecord(ev[0], st);
    st_init(prob, st, -1, 1e-6f, 1e32f, csn);
    cudaEventRecord(ev[1], st);
    for (int i = 0; i < n_iters; ++i) {
      cudaEventRecord(ev[2 + 2 * i], st);
      launch_grid_fused(prob->kind, grid_launch(prob, st), i);
      cudaEventRecord(ev[3 + 2 * i], st);
    }
    cudaEventRecord(ev[2 + 2 * n_iters], st);
    launch_grid_fused_fin(prob->kind, grid_launch(prob, st), n_iters, 0, 0);
    cudaEventRecord(ev[3 + 2 * n_iters], st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_fail(e, "opt_profile_pcg_fused");
  }
  if (status == OPT_OK) {
    float t = 0.f, a = 0.f, f = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    for (int i = 1; i < n_iters; ++i) {
      float x = 0.f;
      cudaEventElapsedTime(&x, ev[2 + 2 * i], ev[3 + 2 * i]);
      a += x;
    }
    cudaEventElapsedTime(&f, ev[2 + 2 * n_iters], ev[3 + 2 * n_iters]);
    ms[0] = t;
    ms[1] = a / (n_iters - 1);
    ms[2] = f;
    prob->pcg_par = n_iters;
    Scalars sc;
    if (cudaMemcpy(&sc, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost) == cudaSuccess) {
      if (sc.timeout) status = OPT_ERR_TIMEOUT;
      else if (sc.misaligned) status = OPT_ERR_CUDA;
    }
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return status;
}

// Vertex-tile tables of the tiled ARAP-mesh apply, built on first use (the
// autotuner, opt_problem_set_apply_form) from the sorted edge list: per tile of
// VT vertices the out-of-tile neighbours (halo), each edge's far end as an
// index into the tile's vertex + halo table, the in-edges arriving from
// outside the tile, the shared-memory slot of every in-edge's J_e p (the
// edge's own slot when it starts inside the tile), and one chunk per tile.
// A tile over the kernel's capacities marks the problem untileable.
static opt_status ensure_tile_tables(opt_problem* q) {
  if (q->d_tchunks) return OPT_OK;
  if (!q->tileable) return OPT_ERR_INVALID_ARG;
  const int V = q->V, E = q->E, nvt = (V + VT - 1) / VT;
  const std::vector<int>& e0 = q->h_e0;
  const std::vector<int>& e1 = q->h_e1;
  std::vector<int> orow((size_t)V + 1, 0), irow((size_t)V + 1, 0), isrc((size_t)E), itpos((size_t)E);
  for (int e = 0; e < E; ++e) {
    orow[(size_t)e0[e] + 1] += 1;
    irow[(size_t)e1[e] + 1] += 1;
  }
  for (int v = 0; v < V; ++v) {
    orow[(size_t)v + 1] += orow[v];
    irow[(size_t)v + 1] += irow[v];
  }
  {
    std::vector<int> fill(irow.begin(), irow.end() - 1);
    for (int e = 0; e < E; ++e) {
      const size_t k = (size_t)fill[e1[e]]++;
      isrc[k] = e0[e];
      itpos[k] = e;
    }
  }
  std::vector<int> hptr((size_t)nvt + 1, 0), rptr((size_t)nvt + 1, 0), hvtx, rin;
  std::vector<int> lnbr((size_t)E, 0), itslot((size_t)E, 0), halo;
  for (int T = 0; T < nvt; ++T) {
    const int vb = T * VT, ve = std::min(V, vb + VT);
    const int eb = orow[vb], ee = orow[ve];
    halo.clear();
    for (int k = eb; k < ee; ++k)
      if (e1[k] < vb || e1[k] >= ve) halo.push_back(e1[k]);
    for (int k = irow[vb]; k < irow[ve]; ++k)
      if (isrc[k] < vb || isrc[k] >= ve) halo.push_back(isrc[k]);
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    if ((int)halo.size() > MT_HALO) {
      q->tileable = false;
      return OPT_ERR_INVALID_ARG;
    }
    auto local = [&](int v) {
      if (v >= vb && v < ve) return v - vb;
      return VT + (int)(std::lower_bound(halo.begin(), halo.end(), v) - halo.begin());
    };
    for (int k = eb; k < ee; ++k) lnbr[k] = local(e1[k]);
    const int nout = ee - eb;
    int nrin = 0;
    for (int i = vb; i < ve; ++i)
      for (int k = irow[i]; k < irow[(size_t)i + 1]; ++k) {
        if (isrc[k] >= vb && isrc[k] < ve) {
          itslot[k] = itpos[k] - eb;
        } else {
          itslot[k] = nout + nrin++;
          rin.push_back((local(isrc[k]) << 16) | (i - vb));
        }
      }
    if (nout + nrin > MT_SLOTS) {
      q->tileable = false;
      return OPT_ERR_INVALID_ARG;
    }
    hvtx.insert(hvtx.end(), halo.begin(), halo.end());
    hptr[(size_t)T + 1] = (int)hvtx.size();
    rptr[(size_t)T + 1] = (int)rin.size();
  }
  std::vector<Chunk> tch;
  for (int T = 0; T < nvt; ++T) tch.push_back(Chunk{0, T * VT, std::min(V, (T + 1) * VT), 0});
  CK(cudaDeviceSynchronize());
  int *dhptr = nullptr, *dhvtx = nullptr, *dlnbr = nullptr, *drptr = nullptr, *drin = nullptr, *ditslot = nullptr;
  CKS(dalloc(q, &dhptr, hptr.size()));
  CKS(upload(dhptr, hptr));
  CKS(dalloc(q, &dhvtx, std::max<size_t>(1, hvtx.size())));
  if (!hvtx.empty()) CKS(upload(dhvtx, hvtx));
  CKS(dalloc(q, &dlnbr, std::max<size_t>(1, lnbr.size())));
  if (E > 0) CKS(upload(dlnbr, lnbr));
  CKS(dalloc(q, &drptr, rptr.size()));
  CKS(upload(drptr, rptr));
  CKS(dalloc(q, &drin, std::max<size_t>(1, rin.size())));
  if (!rin.empty()) CKS(upload(drin, rin));
  CKS(dalloc(q, &ditslot, std::max<size_t>(1, itslot.size())));
  if (E > 0) CKS(upload(ditslot, itslot));
  Chunk* dtch = nullptr;
  CKS(dalloc(q, &dtch, tch.size()));
  CKS(upload(dtch, tch));
  if (tch.size() > (size_t)std::max(q->nvchunks, q->nechunks)) CKS(dalloc(q, &q->d_part, 2 * tch.size()));
  q->d_tchunks = dtch;
  q->ntchunks = (int)tch.size();
  q->h_tch = tch;
  MeshProb& g = q->hm;
  g.hptr = dhptr; g.hvtx = dhvtx; g.lnbr = dlnbr; g.rptr = drptr; g.rin = drin; g.itslot = ditslot;
  g.tchunk_begin = 0;
  g.tchunk_end = q->ntchunks;
  return upload_desc(q, nullptr);
}

// Rebuilds the problem's chunk table with `per` tiles (grid) or vertex tiles
// (graph) per block; 0 restores the default (balanced, 2 blocks per SM for grids, 8 for graphs).
static opt_status rechunk(opt_problem* pb, int per) {
  CK(cudaDeviceSynchronize());
  pb->chunking = per;
  if (pb->gexec) {
    cudaGraphExecDestroy(pb->gexec);
    pb->gexec = nullptr;
    pb->gkey.clear();
  }
  const int bps = per < 0 ? -per : kDefaultBlocksPerSM;     // blocks per SM for balanced splits
  const int target = std::max(1, pb->sms * (is_grid(pb) ? bps : 4 * bps));
  if (is_grid(pb)) {
    std::vector<Chunk> chunks = per > 0 ? make_chunks(pb->ntiles, per, 0)
                                        : make_chunks_balanced(pb->ntiles, target, 0);
    if ((int)chunks.size() > pb->nchunks) {
      CKS(dalloc(pb, &pb->d_chunks, chunks.size()));
      CKS(dalloc(pb, &pb->d_part, 4 * chunks.size()));
    }
    CKS(upload(pb->d_chunks, chunks));
    pb->h_chunks = chunks;
    pb->nchunks = (int)chunks.size();
    pb->hg.chunk_begin = 0;
    pb->hg.chunk_end = pb->nchunks;
  } else {
    const int nvt = (pb->V + VT - 1) / VT;
    std::vector<Chunk> vch = per > 0 ? make_chunks(nvt, per, 0) : make_chunks_balanced(nvt, target, 0);
    for (Chunk& c : vch) { c.begin *= VT; c.end = std::min(pb->V, c.end * VT); }
    std::vector<Chunk> ech = per > 0 ? make_chunks(pb->E, per * VT, 0) : make_chunks_balanced(pb->E, target, 0);
    if ((int)vch.size() > pb->nvchunks) CKS(dalloc(pb, &pb->d_vchunks, vch.size()));
    if ((int)ech.size() > pb->nechunks) CKS(dalloc(pb, &pb->d_echunks, ech.size()));
    const size_t need = 2 * std::max({vch.size(), ech.size(), (size_t)pb->ntchunks});
    if (need > 2 * (size_t)std::max({pb->nvchunks, pb->nechunks, pb->ntchunks})) CKS(dalloc(pb, &pb->d_part, need));
    CKS(upload(pb->d_vchunks, vch));
    CKS(upload(pb->d_echunks, ech));
    pb->h_vch = vch;
    pb->h_ech = ech;
    pb->nvchunks = (int)vch.size();
    pb->nechunks = (int)ech.size();
    pb->hm.vchunk_begin = 0;
    pb->hm.vchunk_end = pb->nvchunks;
    pb->hm.echunk_begin = 0;
    pb->hm.echunk_end = pb->nechunks;
  }
  CKS(upload_desc(pb, nullptr));
  return OPT_OK;
}

opt_status opt_problem_set_chunking(opt_problem* prob, int32_t units_per_block) {
  if (!prob || units_per_block < -64 || units_per_block > 65536) return OPT_ERR_INVALID_ARG;
  return rechunk(prob, units_per_block);
}

// Best granularity of a problem's current layout and apply form: the time of
// one PCG iteration in a short run -- the single-reduction iteration where
// the layout has it (warp and Poisson on 128-pixel tiles), else applyJTJ +
// vector update.
static opt_status tune_granularity(opt_problem* prob, int* best, float* bms) {
  // balanced splits with 1..8 blocks per SM, and fixed runs of 1 and 4 units
  const int cand[] = {-1, -2, -3, -4, -6, -8, 1, 4};
  const bool fused = is_grid(prob) && (prob->kind == K_WARP || prob->kind == K_POISSON) && prob->hg.zb;
  *best = 0;
  *bms = 1e30f;
  for (int c : cand) {
    CKS(rechunk(prob, c));
    float ms[3];
    if (fused) {
      CKS(opt_profile_pcg_fused(prob, 4, nullptr, ms));
      CKS(opt_profile_pcg_fused(prob, 8, nullptr, ms));
    } else {
      CKS(opt_profile_pcg(prob, 4, nullptr, ms));
      CKS(opt_profile_pcg(prob, 8, nullptr, ms));
    }
    const float t = fused ? ms[1] : ms[1] + ms[2];
    if (t < *bms) {
      *bms = t;
      *best = c;
    }
  }
  return rechunk(prob, *best);
}

opt_status opt_problem_autotune(opt_problem* prob, int32_t* chosen, float* best_ms) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  int best = 0;
  float bms = 1e30f;
  if (prob->tileable && ensure_tile_tables(prob) == OPT_OK) {
    // ARAP meshes within the tile capacities: the tiled apply against the two-pass gather
    int b1 = 0, b0 = 0;
    float t1 = 0.f, t0 = 0.f;
    prob->apply_form = 1;
    CKS(tune_granularity(prob, &b1, &t1));
    prob->apply_form = 0;
    CKS(tune_granularity(prob, &b0, &t0));
    prob->apply_form = t1 <= t0 ? 1 : 0;
    best = t1 <= t0 ? b1 : b0;
    bms = std::min(t1, t0);
    CKS(rechunk(prob, best));
  } else {
    CKS(tune_granularity(prob, &best, &bms));
  }
  if (is_grid(prob) && prob->has_grid_desc) {
    // grids: the other tile width, planned afresh from the same descriptor;
    // the faster layout is kept (the handle stays the same)
    opt_solve_params prm;
    opt_solve_params_default(&prm);
    prm.tile_w = prob->tile_w == 128 ? 32 : 128;
    opt_problem* alt = nullptr;
    CKS(opt_problem_create_grid(&prob->grid_desc, &prm, &alt));
    int b2 = 0;
    float t2 = 0.f;
    opt_status st = tune_granularity(alt, &b2, &t2);
    if (st == OPT_OK && t2 < bms) {
      CK(cudaDeviceSynchronize());
      prob->swap_contents(*alt);
      best = b2;
      bms = t2;
    }
    opt_problem_destroy(alt);
    if (st != OPT_OK) return st;
  }
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = bms;
  return OPT_OK;
}

opt_status opt_problem_get_config(const opt_problem* prob, int32_t* tile_w, int32_t* chunking, int32_t* apply_form) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  if (tile_w) *tile_w = is_grid(prob) ? prob->tile_w : 0;
  if (chunking) *chunking = prob->chunking;
  if (apply_form) *apply_form = (prob->d_tchunks || prob->tileable) ? prob->apply_form : -1;
  return OPT_OK;
}

opt_status opt_problem_set_apply_form(opt_problem* prob, int32_t form) {
  if (!prob || form < 0 || form > 1) return OPT_ERR_INVALID_ARG;
  if (form == 1) CKS(ensure_tile_tables(prob));
  CK(cudaDeviceSynchronize());
  if (prob->gexec) {
    cudaGraphExecDestroy(prob->gexec);
    prob->gexec = nullptr;
    prob->gkey.clear();
  }
  prob->apply_form = form;
  return OPT_OK;
}

opt_status opt_eval_energy(opt_problem* prob, double* energy) {
  if (!prob) return OPT_ERR_INVALID_ARG;
  CKS(hook_prepare(prob, 0.0, false));
  CKS(copy_planes_in(prob, prob->x, prob->user_x, prob->nx, nullptr));
  k_reset<<<1, 32>>>(prob->d_s, 1, 0.0);
  st_energy(prob, nullptr, 0, -2);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  Scalars s;
  CK(cudaMemcpy(&s, prob->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  if (energy) *energy = s.E;
  if (s.timeout) return OPT_ERR_TIMEOUT;
  if (s.misaligned) return OPT_ERR_CUDA;
  return s.nonfinite ? OPT_ERR_NUMERIC : OPT_OK;
}

}  // extern "C"
