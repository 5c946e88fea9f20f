// Batched solves: many uneven problems advanced together, one launch per
// phase for the whole batch (the batched precision form of the solver).
//
// The solver kernels already read their problem from a table (probs[chunk.prob])
// and reduce per problem, so a batch is a combined table: every member's
// descriptor (with its own device scalars, vectors and energy history), a
// combined list of tiles (grid) or vertex / edge ranges (graph), and chunks that
// never straddle two problems.  Each phase (PCGInit, applyJTJ, vector update,
// outer update, energies) is one launch per energy kind covering all members;
// members advance in lock-step through the same outer / inner counts, and every
// float64 scalar (alpha, beta, energies, LM damping) stays per problem on the
// device.  The whole batched solve is captured once as a CUDA graph.
//
// The chunk granularity (tiles per chunk) is picked by a small autotuner that
// times one outer iteration of the batch for each candidate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"
#include "opt_launch.h"
#include "opt_problem.h"

using namespace optgb;

namespace {

#define BCK(call)                                              \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      (void)cudaGetLastError();                                \
      return e_ == cudaErrorMemoryAllocation ? OPT_ERR_OOM : OPT_ERR_CUDA; \
    }                                                          \
  } while (0)

struct PlaneCopy {
  const float* src;
  float* dst;
  int rows, cols;
  int src_pitch, dst_pitch;   // in floats
  const int* perm;            // graphs (one row): internal vertex k = caller vertex perm[k]
  int to_caller;              // with perm: 1 = internal -> caller order, 0 = caller -> internal
  int pad;
};

__global__ void k_copy_planes(const PlaneCopy* __restrict__ tab, int n) {
  const PlaneCopy c = tab[blockIdx.y];
  const long long total = (long long)c.rows * c.cols;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    if (c.perm) {
      const int v = c.perm[k];
      if (c.to_caller) c.dst[v] = c.src[k];
      else c.dst[k] = c.src[v];
      continue;
    }
    const int r = (int)(k / c.cols), col = (int)(k - (long long)r * c.cols);
    c.dst[(long long)r * c.dst_pitch + col] = c.src[(long long)r * c.src_pitch + col];
  }
}

__global__ void k_reset_tab(Scalars* const* __restrict__ tab, int n, double lambda0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) scalars_reset(tab[i], lambda0);
}

__global__ void k_lm_decide_tab(Scalars* const* __restrict__ tab, int n, double eta, double lmin, double lmax,
                                double rel_tol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lm_decide(tab[i], eta, lmin, lmax, rel_tol);
}

// Each member's round record (server rounds).
__global__ void k_record_round(Scalars* const* __restrict__ tab, int n, RoundRec* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Scalars* t = tab[i];
  out[i] = RoundRec{t->E, t->E_trial, t->accept, t->outer_done};
}

// Copies every member's scalars and energy history into contiguous buffers.
__global__ void k_gather_results(Scalars* const* __restrict__ tab, double* const* __restrict__ hist, int n,
                                 int hlen, Scalars* __restrict__ s_out, double* __restrict__ h_out) {
  const int i = blockIdx.x;
  if (i >= n) return;
  if (threadIdx.x == 0) s_out[i] = *tab[i];
  for (int k = threadIdx.x; k < hlen; k += blockDim.x) h_out[(long long)i * hlen + k] = hist[i][k];
}

template <class T>
opt_status balloc(std::vector<void*>& allocs, T** ptr, size_t n) {
  void* p = nullptr;
  BCK(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
  allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return OPT_OK;
}

template <class T>
opt_status bupload(std::vector<void*>& allocs, T** ptr, const std::vector<T>& v) {
  opt_status s = balloc(allocs, ptr, v.size());
  if (s != OPT_OK) return s;
  if (!v.empty()) BCK(cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return OPT_OK;
}

struct GridGroup {
  int kind = 0;
  int tw = 32;
  int masked = 0;
  std::vector<int> members;            // indices into opt_batch::probs
  GridProb* d_probs = nullptr;
  Chunk* d_chunks = nullptr;
  int* d_tiles = nullptr;
  double* d_part = nullptr;
  int nchunks = 0;
};

struct MeshGroup {
  int dim = 3;                         // 3: ARAP mesh, 2: warp on a graph, 12: embedded deformation
  int grid3 = 0;                       // volumetric problems (7-point stencil)
  std::vector<int> members;
  MeshProb* d_probs = nullptr;
  Chunk* d_vch = nullptr;
  Chunk* d_ech = nullptr;
  Chunk* d_tch = nullptr;              // tile chunks of the tiled ARAP-mesh apply (NULL: some member untiled)
  double* d_part = nullptr;
  int nv = 0, ne = 0, nt = 0;
};

}  // namespace

struct opt_batch {
  std::vector<opt_problem*> probs;
  std::vector<GridGroup> grids;
  MeshGroup graphs[4];               // [0]: ARAP meshes, [1]: warps on graphs, [2]: volumes,
                                     // [3]: embedded deformation
  int tiles_per_chunk = 0;          // 0 = per-problem default
  std::vector<void*> table_allocs;  // rebuilt with the chunking
  std::vector<void*> allocs;        // fixed for the batch's life
  Scalars** d_stab = nullptr;
  double** d_htab = nullptr;
  PlaneCopy* d_copy_in = nullptr;
  PlaneCopy* d_copy_out = nullptr;
  int ncopy = 0, max_plane = 0;
  Scalars* d_sout = nullptr;
  double* d_hout = nullptr;
  int hcap = 0;
  RoundRec* d_rounds = nullptr;     // server rounds: records, round-major
  int rounds_cap = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  ~opt_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (void* p : table_allocs) cudaFree(p);
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

bool is_grid_kind(int k) { return k == K_WARP || k == K_POISSON; }

// (Re)builds the combined work tables with `tpc` tiles per chunk (0 = each
// member's own chunking).
opt_status build_tables(opt_batch* b, int tpc) {
  cudaDeviceSynchronize();
  for (void* p : b->table_allocs) cudaFree(p);
  b->table_allocs.clear();
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->gkey.clear();
  }
  for (GridGroup& g : b->grids) {
    std::vector<GridProb> gp;
    std::vector<Chunk> chunks;
    std::vector<int> tiles;
    for (size_t mi = 0; mi < g.members.size(); ++mi) {
      opt_problem* pb = b->probs[g.members[mi]];
      const std::vector<int>& t = pb->h_tiles;
      GridProb d = pb->hg;
      d.chunk_begin = (int)chunks.size();
      const int base = (int)tiles.size();
      if (tpc > 0) {
        for (int s = 0; s < pb->ntiles; s += tpc)
          chunks.push_back(Chunk{(int)mi, base + s, base + std::min(s + tpc, pb->ntiles), 0});
      } else {
        // the member's own split: identical reductions to its solo solve
        for (Chunk c : pb->h_chunks) chunks.push_back(Chunk{(int)mi, base + c.begin, base + c.end, 0});
      }
      d.chunk_end = (int)chunks.size();
      tiles.insert(tiles.end(), t.begin(), t.end());
      gp.push_back(d);
    }
    opt_status s;
    if ((s = bupload(b->table_allocs, &g.d_probs, gp)) != OPT_OK) return s;
    if ((s = bupload(b->table_allocs, &g.d_chunks, chunks)) != OPT_OK) return s;
    if ((s = bupload(b->table_allocs, &g.d_tiles, tiles)) != OPT_OK) return s;
    if ((s = balloc(b->table_allocs, &g.d_part, 4 * chunks.size())) != OPT_OK) return s;   // up to 4 partials
    g.nchunks = (int)chunks.size();
  }
  for (MeshGroup& g : b->graphs) {
    if (g.members.empty()) continue;
    std::vector<MeshProb> mp;
    std::vector<Chunk> vch, ech, tch;
    bool tiled = true;
    for (size_t mi = 0; mi < g.members.size(); ++mi) {
      const opt_problem* pm = b->probs[g.members[mi]];
      tiled = tiled && pm->d_tchunks && pm->apply_form;
    }
    for (size_t mi = 0; mi < g.members.size(); ++mi) {
      opt_problem* pb = b->probs[g.members[mi]];
      const std::vector<Chunk>& v = pb->h_vch;
      const std::vector<Chunk>& e = pb->h_ech;
      MeshProb d = pb->hm;
      d.vchunk_begin = (int)vch.size();
      for (Chunk c : v) { c.prob = (int)mi; vch.push_back(c); }
      d.vchunk_end = (int)vch.size();
      d.echunk_begin = (int)ech.size();
      for (Chunk c : e) { c.prob = (int)mi; ech.push_back(c); }
      d.echunk_end = (int)ech.size();
      d.tchunk_begin = (int)tch.size();
      if (tiled) {
        for (Chunk c : pb->h_tch) { c.prob = (int)mi; tch.push_back(c); }
      }
      d.tchunk_end = (int)tch.size();
      mp.push_back(d);
    }
    opt_status s;
    if ((s = bupload(b->table_allocs, &g.d_probs, mp)) != OPT_OK) return s;
    if ((s = bupload(b->table_allocs, &g.d_vch, vch)) != OPT_OK) return s;
    if ((s = bupload(b->table_allocs, &g.d_ech, ech)) != OPT_OK) return s;
    g.d_tch = nullptr;
    if (tiled && (s = bupload(b->table_allocs, &g.d_tch, tch)) != OPT_OK) return s;
    if ((s = balloc(b->table_allocs, &g.d_part, 2 * std::max({vch.size(), ech.size(), tch.size()}))) != OPT_OK)
      return s;
    g.nv = (int)vch.size();
    g.ne = (int)ech.size();
    g.nt = tiled ? (int)tch.size() : 0;
  }
  b->tiles_per_chunk = tpc;
  return OPT_OK;
}

GridLaunch gl(const GridGroup& g, cudaStream_t st) {
  return GridLaunch{g.d_probs, g.d_chunks, g.d_tiles, g.d_part, g.nchunks, st, g.tw, g.masked};
}
MeshLaunch ml(const MeshGroup& g, cudaStream_t st) {
  return MeshLaunch{g.d_probs, g.d_vch, g.d_ech, g.d_part, g.nv, g.ne, st, g.dim, g.grid3, g.d_tch, g.nt};
}

// Uploads the members' descriptors with the solve's flags (outside any capture).
opt_status refresh_descriptors(opt_batch* b, int lm, int use_precond, int outer) {
  for (opt_problem* pb : b->probs) {
    if (pb->Ehist_cap < outer + 1) {
      double* e = nullptr;
      void* p = nullptr;
      BCK(cudaMalloc(&p, sizeof(double) * (outer + 1)));
      pb->allocs.push_back(p);
      pb->pooled.push_back(false);
      e = static_cast<double*>(p);
      pb->d_Ehist = e;
      pb->Ehist_cap = outer + 1;
      if (pb->gexec) {
        cudaGraphExecDestroy(pb->gexec);
        pb->gexec = nullptr;
        pb->gkey.clear();
      }
    }
  }
  for (GridGroup& g : b->grids) {
    std::vector<GridProb> gp(g.members.size());
    BCK(cudaMemcpy(gp.data(), g.d_probs, gp.size() * sizeof(GridProb), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < gp.size(); ++i) {
      opt_problem* pb = b->probs[g.members[i]];
      gp[i].lm = lm;
      gp[i].use_precond = use_precond;
      gp[i].Ehist = pb->d_Ehist;
      gp[i].jtf_out = nullptr;
      gp[i].diag_out = nullptr;
    }
    BCK(cudaMemcpy(g.d_probs, gp.data(), gp.size() * sizeof(GridProb), cudaMemcpyHostToDevice));
  }
  for (MeshGroup& g : b->graphs) {
    if (g.members.empty()) continue;
    std::vector<MeshProb> mp(g.members.size());
    BCK(cudaMemcpy(mp.data(), g.d_probs, mp.size() * sizeof(MeshProb), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < mp.size(); ++i) {
      opt_problem* pb = b->probs[g.members[i]];
      mp[i].lm = lm;
      mp[i].use_precond = use_precond;
      mp[i].Ehist = pb->d_Ehist;
      mp[i].jtf_out = nullptr;
      mp[i].diag_out = nullptr;
    }
    BCK(cudaMemcpy(g.d_probs, mp.data(), mp.size() * sizeof(MeshProb), cudaMemcpyHostToDevice));
  }
  std::vector<double*> ht;
  for (opt_problem* pb : b->probs) ht.push_back(pb->d_Ehist);
  BCK(cudaMemcpy(b->d_htab, ht.data(), ht.size() * sizeof(double*), cudaMemcpyHostToDevice));
  return OPT_OK;
}

void enqueue_copies(opt_batch* b, const PlaneCopy* tab, cudaStream_t st) {
  if (b->ncopy == 0) return;
  const int bx = std::max(1, std::min(64, (b->max_plane + 255) / 256));
  k_copy_planes<<<dim3(bx, b->ncopy), 256, 0, st>>>(tab, b->ncopy);
}

// One outer iteration window [k0, k1) or the whole solve, as stream work.
void enqueue_batch(opt_batch* b, const opt_solve_params& p, bool lm, cudaStream_t st, int outer, bool write_back) {
  const float dmin = (float)p.diag_min, dmax = (float)p.diag_max;
  const int n = (int)b->probs.size();
  enqueue_copies(b, b->d_copy_in, st);
  k_reset_tab<<<(n + 127) / 128, 128, 0, st>>>(b->d_stab, n, lm ? p.lambda0 : 0.0);
  // wide-tile warp groups take the single-reduction PCG iteration when asked
  // for (as a solo solve of each member would), the others the two-pass one
  auto fused = [&](const GridGroup& g) {
    return p.pcg_form == 1 && p.inner > 0 && (g.kind == K_WARP || g.kind == K_POISSON) && g.tw == 128;
  };
  for (int k = 0; k < outer; ++k) {
    // from the second outer iteration on, the wide warps' cos / sin of theta
    // come from the previous outer update
    const int csn_next = k + 1 < outer;
    for (GridGroup& g : b->grids) launch_grid_init(g.kind, gl(g, st), k, dmin, dmax, k > 0);
    for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_init(ml(g, st), k, dmin, dmax);
    for (int i = 0; i < p.inner; ++i) {
      for (GridGroup& g : b->grids) {
        if (fused(g)) launch_grid_fused(g.kind, gl(g, st), i);
        else launch_grid_apply(g.kind, gl(g, st), nullptr, i, 1);
      }
      for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_apply(ml(g, st), nullptr, i, 1);
      for (GridGroup& g : b->grids) if (!fused(g)) launch_grid_update(g.kind, gl(g, st), i);
      for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_update(ml(g, st), i);
    }
    // the single-reduction groups' last step (with x += delta under GN)
    for (GridGroup& g : b->grids)
      if (fused(g)) launch_grid_fused_fin(g.kind, gl(g, st), p.inner, lm ? 0 : 1, lm ? 0 : csn_next);
    if (!lm) {
      for (GridGroup& g : b->grids) if (!fused(g)) launch_grid_step(g.kind, gl(g, st), 0, csn_next);
      for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_step(ml(g, st), 0);
    } else {
      for (GridGroup& g : b->grids) launch_grid_energy(g.kind, gl(g, st), 1, -2);
      for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_energy(ml(g, st), 1, -2);
      k_lm_decide_tab<<<(n + 127) / 128, 128, 0, st>>>(b->d_stab, n, p.eta, p.lambda_min, p.lambda_max, p.rel_tol);
      for (GridGroup& g : b->grids) launch_grid_step(g.kind, gl(g, st), 1, csn_next);
      for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_step(ml(g, st), 1);
    }
  }
  for (GridGroup& g : b->grids) launch_grid_energy(g.kind, gl(g, st), 0, lm ? -1 : outer);
  for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_energy(ml(g, st), 0, lm ? -1 : outer);
  if (write_back) enqueue_copies(b, b->d_copy_out, st);
}

opt_status batch_solve(opt_batch* b, const opt_solve_params* prm_in, opt_report* reports, float* ms_out, bool lm,
                       bool write_back = true) {
  if (!b) return OPT_ERR_INVALID_ARG;
  opt_solve_params p;
  if (prm_in) p = *prm_in;
  else opt_solve_params_default(&p);
  if (p.outer < 1 || p.inner < 0 || p.materialized || p.pcg_form < 0 || p.pcg_form > 1) return OPT_ERR_INVALID_ARG;
  if (lm && (!(p.lambda0 >= 0.0) || !(p.lambda_min <= p.lambda_max) || !(p.diag_min <= p.diag_max)))
    return OPT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)p.stream;
  BCK(cudaStreamSynchronize(st));
  opt_status s = refresh_descriptors(b, lm ? 1 : 0, p.use_precond, p.outer);
  if (s != OPT_OK) return s;
  const int n = (int)b->probs.size();
  const int hlen = p.outer + 1;
  if (b->hcap < hlen) {
    if ((s = balloc(b->allocs, &b->d_hout, (size_t)n * hlen)) != OPT_OK) return s;
    b->hcap = hlen;
  }
  const std::vector<double> key = {double(p.outer), double(p.inner), double(lm), double(p.use_precond), p.lambda0,
                                   p.lambda_min, p.lambda_max, p.diag_min, p.diag_max, p.eta, p.rel_tol,
                                   double(write_back), double(p.pcg_form)};
  if (p.use_graph) {
    if (!b->gexec || key != b->gkey) {
      if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      enqueue_batch(b, p, lm, b->cap_stream, p.outer, write_back);
      const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return OPT_ERR_CUDA;
      }
      const cudaError_t e2 = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) {
        (void)cudaGetLastError();
        return OPT_ERR_CUDA;
      }
      b->gkey = key;
    }
    BCK(cudaEventRecord(b->ev0, st));
    BCK(cudaGraphLaunch(b->gexec, st));
    BCK(cudaEventRecord(b->ev1, st));
  } else {
    BCK(cudaEventRecord(b->ev0, st));
    enqueue_batch(b, p, lm, st, p.outer, write_back);
    BCK(cudaEventRecord(b->ev1, st));
  }
  k_gather_results<<<n, 128, 0, st>>>(b->d_stab, b->d_htab, n, hlen, b->d_sout, b->d_hout);
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(st));
  float ms = 0.f;
  BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  if (ms_out) *ms_out = ms;
  std::vector<Scalars> sv(n);
  std::vector<double> hv((size_t)n * hlen);
  BCK(cudaMemcpy(sv.data(), b->d_sout, n * sizeof(Scalars), cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(hv.data(), b->d_hout, hv.size() * sizeof(double), cudaMemcpyDeviceToHost));
  bool nonfinite = false, timeout = false, misaligned = false;
  for (int i = 0; i < n; ++i) {
    const Scalars& t = sv[i];
    nonfinite |= t.nonfinite != 0;
    timeout |= t.timeout != 0;
    misaligned |= t.misaligned != 0;
    if (!reports) continue;
    opt_report& r = reports[i];
    const int od = lm ? t.outer_done : p.outer;
    r.outer_done = od;
    r.pcg_done = t.pcg_iters;
    r.accepted = lm ? t.accepted_total : p.outer;
    r.converged = t.converged;
    r.E0 = hv[(size_t)i * hlen];
    r.E_final = hv[(size_t)i * hlen + od];
    r.lambda_final = lm ? t.lambda : 0.0;
    if (r.E_history) std::memcpy(r.E_history, &hv[(size_t)i * hlen], sizeof(double) * (od + 1));
    r.ms = ms;
  }
  if (timeout) return OPT_ERR_TIMEOUT;
  if (misaligned) return OPT_ERR_CUDA;
  return nonfinite ? OPT_ERR_NUMERIC : OPT_OK;
}

}  // namespace

extern "C" {

opt_status opt_batch_create(opt_problem* const* probs, int32_t n, opt_batch** out) {
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!probs || n < 1) return OPT_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!probs[i]) return OPT_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n && n <= 4096; ++j)
      if (probs[i] == probs[j]) return OPT_ERR_INVALID_ARG;
  std::unique_ptr<opt_batch> b(new opt_batch());
  b->probs.assign(probs, probs + n);
  // one launch group per (kind, tile width, mask presence): each group runs
  // one kernel variant
  for (int kind : {(int)K_WARP, (int)K_POISSON})
    for (int tw : {32, 128})
      for (int masked : {0, 1}) {
        GridGroup g;
        g.kind = kind;
        g.tw = tw;
        g.masked = masked;
        for (int i = 0; i < n; ++i)
          if (probs[i]->kind == kind && probs[i]->hg.tw == tw && (probs[i]->hg.mask != nullptr) == (masked != 0))
            g.members.push_back(i);
        if (!g.members.empty()) b->grids.push_back(g);
      }
  b->graphs[1].dim = 2;
  b->graphs[2].grid3 = 1;
  b->graphs[3].dim = 12;
  for (int i = 0; i < n; ++i) {
    if (probs[i]->kind == K_MESH) b->graphs[0].members.push_back(i);
    if (probs[i]->kind == K_WARPG) b->graphs[1].members.push_back(i);
    if (probs[i]->kind == K_VOLUME) b->graphs[2].members.push_back(i);
    if (probs[i]->kind == K_EMBED) b->graphs[3].members.push_back(i);
  }
  BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  BCK(cudaEventCreate(&b->ev0));
  BCK(cudaEventCreate(&b->ev1));
  // scalar and history tables, plane copies
  std::vector<Scalars*> stab;
  std::vector<PlaneCopy> cin, cout_;
  int maxp = 0;
  for (opt_problem* pb : b->probs) {
    stab.push_back(pb->d_s);
    for (int c = 0; c < pb->nx; ++c) {
      if (is_grid_kind(pb->kind)) {
        cin.push_back(PlaneCopy{pb->user_x[c], pb->x + c * pb->plane, pb->H, pb->W, pb->W, pb->P, nullptr, 0, 0});
        cout_.push_back(PlaneCopy{pb->x + c * pb->plane, pb->user_x[c], pb->H, pb->W, pb->P, pb->W, nullptr, 0, 0});
      } else {
        cin.push_back(PlaneCopy{pb->user_x[c], pb->x + c * pb->plane, 1, pb->V, pb->V, pb->V, pb->d_perm, 0, 0});
        cout_.push_back(PlaneCopy{pb->x + c * pb->plane, pb->user_x[c], 1, pb->V, pb->V, pb->V, pb->d_perm, 1, 0});
      }
      maxp = std::max<int>(maxp, (int)pb->ulen);
    }
  }
  opt_status s;
  if ((s = bupload(b->allocs, &b->d_stab, stab)) != OPT_OK) return s;
  if ((s = balloc(b->allocs, &b->d_htab, (size_t)n)) != OPT_OK) return s;
  if ((s = bupload(b->allocs, &b->d_copy_in, cin)) != OPT_OK) return s;
  if ((s = bupload(b->allocs, &b->d_copy_out, cout_)) != OPT_OK) return s;
  if ((s = balloc(b->allocs, &b->d_sout, (size_t)n)) != OPT_OK) return s;
  b->ncopy = (int)cin.size();
  b->max_plane = maxp;
  if ((s = build_tables(b.get(), 0)) != OPT_OK) return s;
  *out = b.release();
  return OPT_OK;
}

opt_status opt_batch_destroy(opt_batch* b) {
  if (!b) return OPT_OK;
  cudaDeviceSynchronize();
  delete b;
  return OPT_OK;
}

opt_status opt_batch_set_chunking(opt_batch* b, int32_t tiles_per_chunk) {
  if (!b || tiles_per_chunk < 0 || tiles_per_chunk > 4096) return OPT_ERR_INVALID_ARG;
  return build_tables(b, tiles_per_chunk);
}

opt_status opt_batch_solve_gn(opt_batch* b, const opt_solve_params* params, opt_report* reports, float* ms) {
  return batch_solve(b, params, reports, ms, false);
}

opt_status opt_batch_solve_lm(opt_batch* b, const opt_solve_params* params, opt_report* reports, float* ms) {
  return batch_solve(b, params, reports, ms, true);
}

opt_status opt_batch_autotune(opt_batch* b, const opt_solve_params* params, int32_t* chosen, float* best_ms) {
  if (!b) return OPT_ERR_INVALID_ARG;
  opt_solve_params p;
  if (params) p = *params;
  else opt_solve_params_default(&p);
  p.outer = 1;
  p.inner = std::max(1, std::min(p.inner, 4));
  p.use_graph = 1;
  const int cand[] = {0, 1, 2, 4, 8, 16};
  int best = 0;
  float bms = 1e30f;
  for (int c : cand) {
    opt_status s = build_tables(b, c);
    if (s != OPT_OK) return s;
    float t = 0.f, tmin = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      s = batch_solve(b, &p, nullptr, &t, false, false);
      if (s != OPT_OK && s != OPT_ERR_NUMERIC) return s;
      if (rep > 0) tmin = std::min(tmin, t);
    }
    if (tmin < bms) {
      bms = tmin;
      best = c;
    }
  }
  opt_status s = build_tables(b, best);
  if (s != OPT_OK) return s;
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = bms;
  return OPT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal interface used by the serving engine (serve.cu): one LM outer
// iteration of every member, without energy-history writes, and a gather of
// the members' scalars.
// ---------------------------------------------------------------------------
namespace optgb {

opt_status batch_prepare_round(opt_batch* b, const opt_solve_params& p) {
  return refresh_descriptors(b, 1, p.use_precond, 1);
}

opt_status batch_reserve_rounds(opt_batch* b, int rounds) {
  if (rounds <= b->rounds_cap) return OPT_OK;
  opt_status s = balloc(b->allocs, &b->d_rounds, (size_t)rounds * b->probs.size());
  if (s == OPT_OK) b->rounds_cap = rounds;
  return s;
}

void batch_enqueue_lm_round(opt_batch* b, const opt_solve_params& p, cudaStream_t st, int round) {
  const float dmin = (float)p.diag_min, dmax = (float)p.diag_max;
  const int n = (int)b->probs.size();
  // 128-pixel-tile warp and Poisson groups on the single-reduction iteration
  // when asked for, as in enqueue_batch
  auto fused = [&](const GridGroup& g) {
    return p.pcg_form == 1 && p.inner > 0 && (g.kind == K_WARP || g.kind == K_POISSON) && g.tw == 128;
  };
  for (GridGroup& g : b->grids) launch_grid_init(g.kind, gl(g, st), -2, dmin, dmax, 0);
  for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_init(ml(g, st), -2, dmin, dmax);
  for (int i = 0; i < p.inner; ++i) {
    for (GridGroup& g : b->grids) {
      if (fused(g)) launch_grid_fused(g.kind, gl(g, st), i);
      else launch_grid_apply(g.kind, gl(g, st), nullptr, i, 1);
    }
    for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_apply(ml(g, st), nullptr, i, 1);
    for (GridGroup& g : b->grids) if (!fused(g)) launch_grid_update(g.kind, gl(g, st), i);
    for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_update(ml(g, st), i);
  }
  for (GridGroup& g : b->grids) if (fused(g)) launch_grid_fused_fin(g.kind, gl(g, st), p.inner, 0, 0);
  for (GridGroup& g : b->grids) launch_grid_energy(g.kind, gl(g, st), 1, -2);
  for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_energy(ml(g, st), 1, -2);
  k_lm_decide_tab<<<(n + 127) / 128, 128, 0, st>>>(b->d_stab, n, p.eta, p.lambda_min, p.lambda_max, p.rel_tol);
  for (GridGroup& g : b->grids) launch_grid_step(g.kind, gl(g, st), 1, 0);
  for (const MeshGroup& g : b->graphs) if (!g.members.empty()) launch_mesh_step(ml(g, st), 1);
  if (round < b->rounds_cap)
    k_record_round<<<(n + 127) / 128, 128, 0, st>>>(b->d_stab, n, b->d_rounds + (size_t)round * n);
  k_gather_results<<<n, 128, 0, st>>>(b->d_stab, b->d_htab, n, 0, b->d_sout, b->d_hout);
}

opt_status batch_read_scalars(opt_batch* b, Scalars* host_out, RoundRec* rounds_out, int rounds, cudaStream_t st) {
  const size_t n = b->probs.size();
  BCK(cudaMemcpyAsync(host_out, b->d_sout, n * sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  if (rounds_out && rounds > 0 && rounds <= b->rounds_cap)
    BCK(cudaMemcpyAsync(rounds_out, b->d_rounds, (size_t)rounds * n * sizeof(RoundRec), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  return OPT_OK;
}

}  // namespace optgb
