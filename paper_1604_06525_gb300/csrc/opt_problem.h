// Host-side state of one planned problem (shared by the host translation
// units of the library; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"

// Materialized Jacobian (Sec. 7 "Matrix-free vs. Materialized"): J in CSR over
// the residual rows, and its transpose in CSR over the non-empty unknown
// columns, with the permutation that gathers J's values into J^T's.
struct CsrJ {
  int R = 0;                 // residual rows
  long long nnz = 0;
  int nT = 0;                // unknown columns with at least one entry
  int ngroups = 0;           // residual groups refreshed by evalJ
  int* rp = nullptr;         // R + 1
  int* col = nullptr;        // nnz: internal unknown index
  float* val = nullptr;      // nnz
  int* t_unk = nullptr;      // nT: internal unknown index of each J^T row
  int* t_ptr = nullptr;      // nT + 1
  int* t_row = nullptr;      // nnz: J row of each J^T entry
  int* t_perm = nullptr;     // nnz: index of each J^T entry in val
  float* t_val = nullptr;    // nnz
  float* tvec = nullptr;     // R: t = J p
  double* part = nullptr;    // reduction partials of the J^T pass
  int nblk_t = 0;            // blocks of the J^T pass
  // assembled A = J^T J over the non-empty unknowns (materialized = 2): row k
  // is unknown t_unk[k], columns in the internal unknown index space
  int* a_ptr = nullptr;      // nT + 1
  int* a_col = nullptr;      // nnz_a
  float* a_val = nullptr;    // nnz_a, refreshed once per outer iteration
  long long nnz_a = 0;
};

struct opt_problem {
  int kind = 0;
  int nx = 0;             // unknown planes
  int nm = 0;             // distinct-diagonal planes
  int sms = 148;
  // grid
  int W = 0, H = 0, P = 0;
  // graph
  int V = 0, E = 0;
  long long plane = 0;    // internal plane stride (P*H or Vp)
  long long ulen = 0;     // caller plane length (W*H or V)
  optgb::GridProb hg{};
  optgb::GridProb* dg = nullptr;
  optgb::Chunk* d_chunks = nullptr;
  int nchunks = 0;
  int* d_tiles = nullptr;
  int ntiles = 0;
  optgb::MeshProb hm{};
  optgb::MeshProb* dm = nullptr;
  optgb::Chunk* d_vchunks = nullptr;
  optgb::Chunk* d_echunks = nullptr;
  int nvchunks = 0, nechunks = 0;
  optgb::Chunk* d_tchunks = nullptr;   // tiled ARAP-mesh apply: one chunk per vertex tile (NULL: untiled)
  int ntchunks = 0;
  bool tileable = false;                // an ARAP mesh the tiled apply may take (tables built on first use)
  int apply_form = 0;                   // ARAP meshes: 1 tiled apply, 0 two-pass gather (the default)
  int chunking = 0;                     // the granularity last set (0 = default)
  int tile_w = 0;                       // grids: tile width (32 or 128)
  bool has_grid_desc = false;           // grids: the planning input, kept for re-planning at another
  opt_grid_desc grid_desc{};            //   tile width (its arrays are the caller's and outlive the problem)
  // host mirrors of the work tables (batches build their combined tables from these)
  std::vector<int> h_tiles;
  std::vector<optgb::Chunk> h_chunks, h_vch, h_ech, h_tch;
  // host copies kept for building the materialized Jacobian
  std::vector<unsigned char> h_mask;    // grid mask (empty = none)
  std::vector<int> h_hpix;              // grid handles (pitched index) / mesh handles (vertex)
  std::vector<int> h_e0, h_e1;          // sorted edges (internal vertex order)
  int* d_perm = nullptr;                // graphs: internal vertex k is the caller's vertex d_perm[k]
  CsrJ csr;
  // common
  double* d_part = nullptr;
  optgb::Scalars* d_s = nullptr;
  double* d_Ehist = nullptr;
  int Ehist_cap = 0;
  float* user_x[12] = {};
  float* d_tmp = nullptr;     // nx planes: caller p (apply hook)
  float* d_jtf = nullptr;     // nx planes: J^T F (hook)
  float* d_diag = nullptr;    // nm planes: diag (hook)
  float* x = nullptr;
  float* pbuf = nullptr;
  float* dvec = nullptr;
  float* rvec = nullptr;
  float* qvec = nullptr;
  std::vector<void*> allocs;
  std::vector<bool> pooled;             // allocs[k] came from the library's stream-ordered pool
  int pcg_par = 0;
  // persistent PCG loop (wide warps): grid barrier state and the number of
  // blocks that can be resident at once (0 = not available)
  optgb::GridBarrier* d_gbar = nullptr;
  int coop_cap = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // Exchanges everything two problems hold (the autotuner keeps a layout
  // planned afresh under the caller's handle).  Member by member, so every
  // device allocation, stream, event and graph keeps exactly one owner.
  void swap_contents(opt_problem& o) {
    using std::swap;
    swap(kind, o.kind); swap(nx, o.nx); swap(nm, o.nm); swap(sms, o.sms);
    swap(W, o.W); swap(H, o.H); swap(P, o.P); swap(V, o.V); swap(E, o.E);
    swap(plane, o.plane); swap(ulen, o.ulen);
    swap(hg, o.hg); swap(dg, o.dg); swap(d_chunks, o.d_chunks); swap(nchunks, o.nchunks);
    swap(d_tiles, o.d_tiles); swap(ntiles, o.ntiles);
    swap(hm, o.hm); swap(dm, o.dm); swap(d_vchunks, o.d_vchunks); swap(d_echunks, o.d_echunks);
    swap(nvchunks, o.nvchunks); swap(nechunks, o.nechunks); swap(d_tchunks, o.d_tchunks);
    swap(ntchunks, o.ntchunks); swap(tileable, o.tileable); swap(apply_form, o.apply_form); swap(chunking, o.chunking);
    swap(tile_w, o.tile_w); swap(has_grid_desc, o.has_grid_desc); swap(grid_desc, o.grid_desc);
    swap(h_tiles, o.h_tiles); swap(h_chunks, o.h_chunks); swap(h_vch, o.h_vch); swap(h_ech, o.h_ech);
    swap(h_tch, o.h_tch);
    swap(h_mask, o.h_mask); swap(h_hpix, o.h_hpix); swap(h_e0, o.h_e0); swap(h_e1, o.h_e1);
    swap(d_perm, o.d_perm); swap(csr, o.csr);
    swap(d_part, o.d_part); swap(d_s, o.d_s); swap(d_Ehist, o.d_Ehist); swap(Ehist_cap, o.Ehist_cap);
    swap(user_x, o.user_x); swap(d_tmp, o.d_tmp); swap(d_jtf, o.d_jtf); swap(d_diag, o.d_diag);
    swap(x, o.x); swap(pbuf, o.pbuf); swap(dvec, o.dvec); swap(rvec, o.rvec); swap(qvec, o.qvec);
    swap(allocs, o.allocs); swap(pooled, o.pooled); swap(pcg_par, o.pcg_par);
    swap(d_gbar, o.d_gbar); swap(coop_cap, o.coop_cap); swap(cap_stream, o.cap_stream);
    swap(gexec, o.gexec); swap(gkey, o.gkey); swap(ev0, o.ev0); swap(ev1, o.ev1);
  }

  ~opt_problem() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (size_t k = 0; k < allocs.size(); ++k) {
      if (k < pooled.size() && pooled[k]) cudaFreeAsync(allocs[k], nullptr);
      else cudaFree(allocs[k]);
    }
  }
};

struct opt_batch;

namespace optgb {
// api.cu: records a failed CUDA call for opt_last_error (OOM or CUDA status)
opt_status cuda_fail(cudaError_t e, const char* what);
// batch.cu (serving engine interface)
// What a server round leaves of each member after its LM decision: the
// energy at the start of the round, the trial energy, the decision and the
// outer iterations done.
struct RoundRec {
  double E, E_trial;
  int accept, outer_done;
};
opt_status batch_prepare_round(opt_batch* b, const opt_solve_params& p);
// Room for `rounds` rounds of records (one RoundRec per member and round).
opt_status batch_reserve_rounds(opt_batch* b, int rounds);
// One LM outer iteration of every member; the records of round `round` (of
// the reserved ones) are written at its end.
void batch_enqueue_lm_round(opt_batch* b, const opt_solve_params& p, cudaStream_t st, int round);
// Copies the members' scalars and the records of the first `rounds` rounds
// (round-major) to the host; synchronises the stream.
opt_status batch_read_scalars(opt_batch* b, Scalars* host_out, RoundRec* rounds_out, int rounds, cudaStream_t st);
// api.cu: caller planes (dense rows for grids, caller vertex order for
// graphs) <-> internal planes
opt_status copy_planes_in(const opt_problem* pb, float* internal, float* const* user, int n, cudaStream_t st);
opt_status copy_planes_out(const opt_problem* pb, float* const* user, const float* internal, int n,
                           cudaStream_t st);
// materialize.cu
opt_status csr_build(opt_problem* pb, int mode);   // mode 1: J and J^T; mode 2: also the pattern of J^T J
void csr_evalj(opt_problem* pb, cudaStream_t st, int mode);
void csr_apply(opt_problem* pb, cudaStream_t st, int par, int mode);
}  // namespace optgb
