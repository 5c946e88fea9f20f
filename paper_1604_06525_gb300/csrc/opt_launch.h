// Host-side launch descriptors and launchers of the solver kernels.
#pragma once

#include "opt_internal.cuh"

namespace optgb {

struct GridLaunch {
  const GridProb* probs;
  const Chunk* chunks;
  const int* tiles;
  double* part;
  int nchunks;
  cudaStream_t stream;
  int tw;        // tile width of every problem in the launch (32 or 128)
  int masked;    // every problem in the launch has a mask (wide warp kernel variant)
};

struct MeshLaunch {
  const MeshProb* probs;
  const Chunk* vchunks;
  const Chunk* echunks;
  double* part;
  int nvchunks, nechunks;
  cudaStream_t stream;
  int dim;       // 3: ARAP mesh (6 unknowns per vertex); 2: warp on a graph (3 unknowns);
                 // 12: embedded deformation (12 unknowns)
  int grid3;     // dim 3 on a W x H x D voxel grid: neighbours from the 7-point stencil, not the lists
  const Chunk* tchunks;   // one chunk per vertex tile (tiled ARAP-mesh apply), NULL if not every problem is tiled
  int ntchunks;
};

// Launches kernel k with programmatic stream serialization (the kernel must
// begin with pdl_begin()).  Works inside stream capture as well.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// grid_kernels.cu
cudaError_t grid_kernels_prepare();   // one-time kernel attributes (call outside capture)
// csn_in (wide warps): PCGInit reads cos / sin of theta from the planes an
// outer update (csn_out) or launch_grid_csn wrote instead of evaluating them
void launch_grid_init(int kind, const GridLaunch& L, int k_outer, float dmin, float dmax, int csn_in);
void launch_grid_apply(int kind, const GridLaunch& L, const float* p_override, int par, int update);
void launch_grid_update(int kind, const GridLaunch& L, int par);
void launch_grid_energy(int kind, const GridLaunch& L, int mode, int hist_idx);
// Single-reduction PCG (warp or Poisson on 128-pixel tiles; problems planned
// with z / w buffers): iteration `it` (0 starts from r_0, M^-1), and the
// pending step of the last iteration (p of parity par = the iteration count);
// step = 1 also applies the Gauss-Newton update x += delta (csn_out, warp:
// and cos / sin of theta)
void launch_grid_fused(int kind, const GridLaunch& L, int it);
void launch_grid_fused_fin(int kind, const GridLaunch& L, int par, int step, int csn_out);
void launch_grid_step(int kind, const GridLaunch& L, int cond, int csn_out);
// cos / sin of theta at the current unknowns into the cos / sin planes (wide warps)
void launch_grid_csn(const GridLaunch& L);
// Poisson, tile width 128: the degree plane the wide kernels read (S_i + 1 on
// free pixels, 0 elsewhere; pitched like the mask, P x H bytes)
void launch_pois_sdeg(int W, int H, int P, const uint8_t* mask, uint8_t* out, cudaStream_t st);
// Persistent PCG loop (wide warp tiles only): the largest chunk count whose
// blocks are all resident at once (0 if unknown), and the cooperative launch
// of n_inner PCG iterations (applyJTJ + update) starting at parity par0.
int grid_coop_capacity(int masked);
cudaError_t launch_grid_pcg_coop(const GridLaunch& L, GridBarrier* gb, int par0, int n_inner);
// bounded staging-wait self-test (complete = 0: the wait runs out)
cudaError_t launch_staging_selftest(int complete, unsigned long long limit_ns, int* out, cudaStream_t st);
cudaError_t launch_barrier_selftest(GridBarrier* gb, int nblocks, unsigned int expected, int rounds,
                                    unsigned long long limit_ns, cudaStream_t st);

// graph_kernels.cu
void launch_mesh_init(const MeshLaunch& L, int k_outer, float dmin, float dmax);
void launch_mesh_apply(const MeshLaunch& L, const float* p_override, int par, int update);
void launch_mesh_update(const MeshLaunch& L, int par);
void launch_mesh_energy(const MeshLaunch& L, int mode, int hist_idx);
void launch_mesh_step(const MeshLaunch& L, int cond);

// graph2d_kernels.cu (dim == 2; reached through the launch_mesh_* functions)
void launch_wg_init(const MeshLaunch& L, int k_outer, float dmin, float dmax);
void launch_wg_apply(const MeshLaunch& L, const float* p_override, int par, int update);
void launch_wg_update(const MeshLaunch& L, int par);
void launch_wg_energy(const MeshLaunch& L, int mode, int hist_idx);
void launch_wg_step(const MeshLaunch& L, int cond);

// embedded_kernels.cu (dim == 12; reached through the launch_mesh_* functions)
void launch_ed_init(const MeshLaunch& L, int k_outer, float dmin, float dmax);
void launch_ed_apply(const MeshLaunch& L, const float* p_override, int par, int update);
void launch_ed_update(const MeshLaunch& L, int par);
void launch_ed_energy(const MeshLaunch& L, int mode, int hist_idx);
void launch_ed_step(const MeshLaunch& L, int cond);

}  // namespace optgb
