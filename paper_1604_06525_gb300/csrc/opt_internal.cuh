// Internal definitions shared by the CUDA translation units of the solver.
//
// Data layout in HBM (struct of arrays, float32):
//  * grid problems keep every plane pitched: row pitch P = W rounded up to the
//    tile width (32 or 128 floats), plane stride P*H; tiles are tw x TH pixels
//    (tw = 32, or 128 for wide warps); the 32-wide kernels walk a 128-wide
//    tile as four 32 x 8 sub-tiles;
//  * graph problems keep vertex planes of stride Vp = V rounded up to 32;
//  * the PCG vectors delta, r, p, q have one plane per unknown component; the
//    inverse Jacobi preconditioner M^-1 (and the LM damping diagonal D) keep
//    one plane per *distinct* diagonal: the x/y (x/y/z) displacement rows of a
//    pixel (vertex) always share their diagonal entry.
//
// Work is described by a chunk table: one CUDA block per chunk, a chunk is a
// run of tiles (grid) or of vertices / edges (graph) of ONE problem, so the
// same kernels serve a single solve and a batch of uneven problems.
//
// Reductions (p.q, r.z, energies) carry float64 accuracy from the first term
// on: each thread accumulates its terms as a compensated float32 pair (every
// product split exactly by one FMA, every addition made error-free by TwoSum:
// Ogita, Rump & Oishi's Dot2, see F2 below), warps combine the pairs in a fixed
// shuffle order, each warp's pair becomes a float64 hi + lo, and float64 takes
// over from there (the float64 pipe of this part is narrow, so it is kept to
// the last levels).  Each block writes its partial to a per-chunk slot, and the
// last block of a problem to arrive (atomic counter) sums the problem's
// partials in chunk order in float64, so the result does not depend on block
// scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace optgb {

// K_WARPG: the warp on a graph; K_VOLUME: volumetric ARAP (the mesh energy on a voxel grid);
// K_EMBED: embedded deformation (12 unknowns per vertex)
enum Kind : int { K_WARP = 0, K_POISSON = 1, K_MESH = 2, K_WARPG = 3, K_VOLUME = 4, K_EMBED = 5 };

constexpr int TW = 32;            // grid tile width  (pixels)
constexpr int TH = 8;             // grid tile height (pixels)
constexpr int NT = 256;           // threads per block (grid and graph kernels)
constexpr int HW = TW + 2;        // staged halo width
constexpr int HH = TH + 2;        // staged halo height
// 128-pixel tiles: the staged box of a float plane (columns x0 - 4 .. x0 + 131)
// and of the byte plane (columns x0 - 16 .. x0 + 143), HH rows each
constexpr int WIDE_BOX_W = 136;
constexpr int WIDE_BYTE_BOX_W = 160;
constexpr int VT = 256;           // vertices per vertex tile (graph)
// capacities of the tiled ARAP-mesh apply (one tile of VT vertices per pass):
// out-of-tile neighbours staged with the tile, and J_e p slots (the tile's
// out-edges plus its in-edges that start outside the tile)
constexpr int MT_HALO = 384;
constexpr int MT_SLOTS = 2304;

// Device-resident scalars of one problem.  Written only by the single
// finishing block of a reduction or by the one-thread LM decision kernel.
struct __align__(16) Scalars {
  double rz;          // r.z of the current PCG iterate
  double pq;          // p.q of the current PCG iteration
  double E;           // E(x) at the current outer iteration
  double E_trial;     // E(x + delta)            (LM)
  double model;       // |F(x) + J(x) delta|^2   (LM)
  double lambda;      // LM damping
  double nu;          // LM damping growth factor
  double part0;       // partial sum handed from a first graph pass to the second
  double part1;
  float alpha_f;      // alpha = rz / pq, rounded once to float
  float beta_f;       // beta  = rz' / rz
  float lambda_f;
  float pad0;
  int pcg_active;     // 0 once PCG broke down (rz == 0 or pq <= 0)
  int pcg_iters;      // completed PCG iterations in the current solve
  int accept;         // LM: the last trial step was accepted
  int done;           // LM: converged, later kernels of the solve skip work
  int accepted_total;
  int outer_done;
  int converged;
  int nonfinite;      // a non-finite scalar was produced
  unsigned int counter;   // last-block counter
  unsigned int timeout;   // a bounded wait for a tensor copy ran out (the solve reports OPT_ERR_TIMEOUT)
  unsigned int misaligned;  // a staging area could not take tensor copies (the solve reports OPT_ERR_CUDA)
  unsigned int pad1;
  double alpha_d;     // float64 solver: alpha = rz / pq
  double beta_d;      // float64 solver: beta  = rz' / rz
};

struct Chunk {
  int prob;           // problem index
  int begin, end;     // tile (grid) / vertex / edge range
  int pad;
};

// Grid problem (image warping, Poisson).  Pointers are device pointers.
struct GridProb {
  int kind, W, H, P;
  int tw;                       // tile width: 32 or 128 pixels (tiles are tw x TH)
  int ntx, nty;                 // tiles per row / column
  long long plane;              // P * H
  int chunk_begin, chunk_end;   // this problem's chunks (for the final reduction)
  float s_w, s_f, w_reg, w_fit;
  int use_precond, lm;
  float* x;                     // unknown planes (working copy)
  const float* c;               // constant planes (UrShape or guidance)
  const uint8_t* mask;          // pitched mask, NULL = none
  const uint8_t* sdeg;          // Poisson, tw = 128: degree plane (S_i + 1 on free pixels, 0 elsewhere)
  // Poisson, tw = 128, masked: quads holding a free pixel, one 32-bit word per
  // (row, tile column), bit l for the quad at x = 128 tx + 4 l (NULL: all);
  // the vector update skips the others
  const unsigned int* live;
  // tw = 128: tensor maps (CUtensorMap, 128 bytes each) of the planes the wide
  // kernels stage: [0] the float slab (3-D: P x H x planes), [1] the unknowns
  // (3-D: P x H x nx), [2] the byte plane (2-D: mask, or the Poisson degree
  // plane; absent for an unmasked warp); NULL: staged with cp.async
  const unsigned long long* tmap;
  // slab plane index (6 bits each) of r, M^-1, p (parity 0), cos / sin and
  // the constants: zpack = z_r | z_m << 6 | z_p << 12 | z_csn << 18 | z_c << 24
  int zpack;
  // warp, tw = 128: the single-reduction PCG iteration's double-buffered
  // z = M^-1 r and w = M^-1 q (3 planes per buffer, buffer 1 at + 3 planes;
  // NULL where the problem has none) and their slab plane indices
  // (zpack2 = z_z | z_w << 6)
  float *zb, *wb;
  int zpack2;
  float *d, *r, *p, *q;         // PCG vectors
  float *m, *dc;                // M^-1 and LM diagonal (distinct-diagonal planes)
  float* csn;                   // warp, tw = 128: cos / sin of theta (2 planes, written by PCGInit)
  const int* hbeg;              // per tile id: first handle (ntx*nty + 1 entries)
  const int* hpix;              // handle pixel index y*P + x, sorted by tile
  const float* htgt;            // handle target displacement (2 per handle)
  float* jtf_out;               // optional J^T F output planes (parity hook)
  float* diag_out;              // optional diag(J^T J) output planes (distinct)
  Scalars* s;
  double* Ehist;
};

// Graph problem (ARAP mesh).
struct MeshProb {
  int V, E, Vp, pad;
  int gw, gh, gd, gpad;         // volumetric problems: voxel grid W x H x D (0 for graphs)
  int vchunk_begin, vchunk_end;
  int echunk_begin, echunk_end;
  int tchunk_begin, tchunk_end; // tiled apply: this problem's vertex tiles in the tile-chunk table
  float s_w, s_f, w_reg, w_fit;
  float s_r, w_rot;             // embedded deformation: column constraint weight
  int use_precond, lm;
  float* x;                     // 6 planes: displacement, angles (embedded deformation: 12)
  const float* U;               // 3 planes
  const float* degw;            // w_reg * (outdeg + indeg) + w_fit[handle]
  const int* e0;                // edges sorted by (v0, v1)
  const int* e1;
  const int* orow;              // V + 1: out-edges of v are e1[orow[v] .. orow[v+1])
  const int* irow;              // V + 1: in-edges of v come from isrc[irow[v] .. irow[v+1])
  const int* isrc;              // E: sources of the in-edges, ascending per vertex
  // vertex-tile tables of the tiled apply (NULL: the problem exceeds the
  // capacities above and uses the general path)
  const int* hptr;              // tiles + 1: the halo of tile T is hvtx[hptr[T] .. hptr[T+1])
  const int* hvtx;              // out-of-tile vertices adjacent to the tile, ascending
  const int* lnbr;              // E: each edge's far end as an index into its tile's vertex + halo table
  const int* rptr;              // tiles + 1: in-edges from outside tile T are rin[rptr[T] .. rptr[T+1])
  const int* rin;               // (source table index << 16) | target index within the tile
  const int* itslot;            // E: shared-memory slot of each in-edge's J_e p (irow order)
  float *d, *r, *p, *q;         // 6 planes each
  float *m, *dc;                // 4 planes: displacement, ax, ay, az
  float4* grec;                 // 3 float4 per vertex: U, cos / sin of the angles (PCGInit)
  float4* vrec;                 // 2 float4 per vertex: x (PCGInit) or p (applyJTJ)
  const int* hbeg;              // per vertex tile: first handle
  const int* hpix;              // handle vertex, sorted
  const float* htgt;            // 3 per handle
  float* jtf_out;
  float* diag_out;
  Scalars* s;
  double* Ehist;
};

// ---------------------------------------------------------------------------
// programmatic dependent launch
// ---------------------------------------------------------------------------
// Every solver kernel is launched with programmatic stream serialization
// (launch_pdl), so the launch of the next kernel of the chain overlaps the end
// of this one.  Each kernel calls pdl_begin() before it reads or writes
// anything a solver kernel writes: it waits until the kernel before it has
// completed and its writes are visible.  The grid kernels read their work
// chunk and problem descriptor (written only by the host, before the launch)
// ahead of it, overlapping those loads with the previous kernel's tail.  By default a kernel's dependents launch as its blocks exit;
// the graph kernels release them earlier with pdl_trigger() once the block's
// main pass is over (measured: 5% faster for the mesh, slower for the grid
// kernels, whose blocks would crowd onto the SMs that free up first).
// Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// grid-wide barrier of a cooperative launch (all blocks co-resident)
// ---------------------------------------------------------------------------
// Every wait is bounded: a block that has waited longer than limit_ns sets
// `timeout` and the barrier reports failure, so the kernel returns instead
// of hanging; the host turns the flag into OPT_ERR_TIMEOUT.  count returns to
// 0 at every completed barrier; the host clears the struct before a launch.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int timeout;
  int pad;
};

constexpr unsigned long long kBarrierLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Must be called by every thread of every block of the launch; `expected` is
// the number of blocks that take part (gridDim.x).  Returns false on timeout.
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned int expected,
                                          unsigned long long limit_ns = kBarrierLimitNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_u32(&gb->gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u) + 1u;
    if (arrived == expected) {
      gb->count = 0u;
      __threadfence();
      st_release_u32(&gb->gen, g + 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(&gb->gen) == g) {
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&gb->timeout, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of a and b over the block; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[NT / 32], sb[NT / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = l < NT / 32 ? sa[l] : 0.0;
    b = l < NT / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// ---------------------------------------------------------------------------
// compensated float32 accumulation (error-free transformations)
// ---------------------------------------------------------------------------
// A sum is held as the unevaluated pair hi + lo of float32 values.  A product
// x * y enters exactly: p = fl(x * y) and e = fma(x, y, -p) satisfy p + e =
// x * y (TwoProduct); an addend enters through Knuth's TwoSum, which returns
// the rounded sum and its exact rounding error, and the errors are collected
// in lo.  This is the Sum2 / Dot2 scheme of Ogita, Rump & Oishi ("Accurate sum
// and dot product", SIAM J. Sci. Comput. 26(6), 2005): the result is as
// accurate as if accumulated in twice the float32 precision (~48 bits), on
// par with float64 accumulation, at float32 issue rates.  Every operation is
// an explicitly rounded intrinsic, so the compiler can neither contract nor
// reorder it (either would destroy the error terms).
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_zero() { return F2{0.f, 0.f}; }

// hi += x exactly, the rounding error goes to lo (TwoSum, 6 additions)
__device__ __forceinline__ void f2_add(F2& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float z = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(x, z));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}

// a += x * y with the product split exactly (TwoProduct) before the TwoSum
__device__ __forceinline__ void f2_add_prod(F2& a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  f2_add(a, p);
  a.lo = __fadd_rn(a.lo, e);
}

// a += b for two pairs
__device__ __forceinline__ void f2_add_f2(F2& a, F2 b) {
  f2_add(a, b.hi);
  a.lo = __fadd_rn(a.lo, b.lo);
}

__device__ __forceinline__ double f2_to_double(F2 a) { return (double)a.hi + (double)a.lo; }

// Two compensated pairs side by side (lanes x and y), advanced by the packed
// float32 pair instructions of this architecture: one instruction serves both
// lanes, and each lane runs exactly the scalar F2 arithmetic above.
struct F2x2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ F2x2 f2x2_zero() {
  return F2x2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
}
__device__ __forceinline__ void f2x2_add(F2x2& a, float2 x) {
  const float2 s = pk_add(a.hi, x);
  const float2 z = pk_sub(s, a.hi);
  const float2 e = pk_add(pk_sub(a.hi, pk_sub(s, z)), pk_sub(x, z));
  a.hi = s;
  a.lo = pk_add(a.lo, e);
}
__device__ __forceinline__ void f2x2_add_prod(F2x2& a, float2 x, float2 y) {
  const float2 p = pk_mul(x, y);
  const float2 e = pk_fma(x, y, make_float2(-p.x, -p.y));
  f2x2_add(a, p);
  a.lo = pk_add(a.lo, e);
}
// the two lanes combined into one pair
__device__ __forceinline__ F2 f2x2_fold(const F2x2& a) {
  F2 r{a.hi.x, a.lo.x};
  f2_add_f2(r, F2{a.hi.y, a.lo.y});
  return r;
}

// Sum of a pair over the warp (fixed shuffle order); valid in lane 0.
__device__ __forceinline__ F2 warp_sum_f2(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F2 w;
    w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    f2_add_f2(v, w);
  }
  return v;
}

// Block sum of per-thread compensated pairs: pairs within each warp, float64
// across the warps; the result is valid in thread 0.  Called once per kernel
// (its shared slots are not reused).
__device__ __forceinline__ void block_sum2f(F2 a, F2 b, double& ra, double& rb) {
  __shared__ double sa[NT / 32], sb[NT / 32];
  a = warp_sum_f2(a);
  b = warp_sum_f2(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = f2_to_double(a); sb[w] = f2_to_double(b); }
  __syncthreads();
  ra = 0.0;
  rb = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) { ra += sa[k]; rb += sb[k]; }
  }
}

// Stores this chunk's two partial sums and reports whether this block is the
// last of its problem to do so.  Must be called by every thread of the block.
__device__ __forceinline__ bool publish_partials(double* part, int chunk, F2 fa, F2 fb,
                                                 unsigned int* counter, unsigned int nchunks) {
  __shared__ int s_last;
  double a, b;
  block_sum2f(fa, fb, a, b);
  if (threadIdx.x == 0) {
    __stcg(&part[2 * chunk], a);
    __stcg(&part[2 * chunk + 1], b);
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == nchunks - 1);
  }
  __syncthreads();
  return s_last != 0;
}

// In the last block: sums partials [cb, ce) in chunk order (thread-strided,
// then a fixed tree) and resets the counter.  Result valid in thread 0.
__device__ __forceinline__ void gather_partials(const double* part, int cb, int ce,
                                                unsigned int* counter, double& a, double& b) {
  __threadfence();
  a = 0.0;
  b = 0.0;
#pragma unroll 4
  for (int c = cb + (int)threadIdx.x; c < ce; c += NT) {
    a += __ldcg(&part[2 * c]);
    b += __ldcg(&part[2 * c + 1]);
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) *counter = 0u;
}

// Four partial sums per chunk (the single-reduction PCG iteration): as
// publish_partials / gather_partials, with slots part[4 * chunk + 0..3] (the
// grid problems' partial buffers hold four doubles per chunk).
__device__ __forceinline__ bool publish_partials4(double* part, int chunk, const F2 (&f)[4],
                                                  unsigned int* counter, unsigned int nchunks) {
  __shared__ double s4[4][NT / 32];
  __shared__ int s_last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const F2 v = warp_sum_f2(f[k]);
    if (l == 0) s4[k][w] = f2_to_double(v);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double a = 0.0;
#pragma unroll
    for (int j = 0; j < NT / 32; ++j) a += s4[threadIdx.x][j];
    __stcg(&part[4 * chunk + threadIdx.x], a);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == nchunks - 1);
  }
  __syncthreads();
  return s_last != 0;
}

// In the last block: the four sums over chunks [cb, ce) in chunk order
// (thread-strided, then a fixed tree); valid in thread 0; resets the counter.
__device__ __forceinline__ void gather_partials4(const double* part, int cb, int ce, unsigned int* counter,
                                                 double (&out)[4]) {
  __shared__ double g4[4][NT / 32];
  __threadfence();
  double a[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
  for (int c = cb + (int)threadIdx.x; c < ce; c += NT) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += __ldcg(&part[4 * c + k]);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = warp_sum(a[k]);
    if (l == 0) g4[k][w] = a[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      out[k] = 0.0;
      for (int j = 0; j < NT / 32; ++j) out[k] += g4[k][j];
    }
    *counter = 0u;
  }
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// Fresh scalars for a solve: zero iterates and counters, LM damping lambda0,
// growth factor 2.
__device__ __forceinline__ void scalars_reset(Scalars* s, double lambda0) {
  Scalars z;
  memset(&z, 0, sizeof(z));
  z.lambda = lambda0;
  z.lambda_f = (float)lambda0;
  z.nu = 2.0;
  *s = z;
}

// LM decision after the trial energy (Sec. 4 LM; Nielsen's damping update,
// Madsen, Nielsen & Tingleff 2004, Sec. 3.2): gain ratio rho = (E - E') /
// (E - |F + J d|^2); accept if rho > eta with lambda *= max(1/3, 1 - (2 rho -
// 1)^3) and nu = 2, else lambda *= nu and nu *= 2; lambda clamped to
// [lmin, lmax].  An accepted step whose relative energy change is below
// rel_tol (> 0) ends the solve.  Every decision counts as an outer iteration.
__device__ __forceinline__ void lm_decide(Scalars* t, double eta, double lmin, double lmax, double rel_tol) {
  if (t->done) {
    t->accept = 0;
    return;
  }
  const double E = t->E, Et = t->E_trial;
  const double pred = E - t->model;
  const double rho = pred > 0.0 ? (E - Et) / pred : -INFINITY;
  double lam = t->lambda;
  t->outer_done += 1;
  if (rho > eta) {
    const double u = 2.0 * rho - 1.0;
    lam *= fmax(1.0 / 3.0, 1.0 - u * u * u);
    t->nu = 2.0;
    t->accept = 1;
    t->accepted_total += 1;
    if (rel_tol > 0.0 && (Et == 0.0 || fabs(E - Et) / E < rel_tol)) {
      t->done = 1;
      t->converged = 1;
    }
  } else {
    lam *= t->nu;
    t->nu *= 2.0;
    t->accept = 0;
  }
  lam = fmin(fmax(lam, lmin), lmax);
  t->lambda = lam;
  t->lambda_f = (float)lam;
  if (!isfinite(Et) && t->accept) t->nonfinite = 1;
}

// Inverse Jacobi preconditioner entry for diagonal `dg` with LM damping
// lambda * clamp(dg): 1 / (dg + lambda * Dc); rows with a zero diagonal get 1.
__device__ __forceinline__ float minv_entry(float dg, float lam, float dmin, float dmax,
                                            int use_precond, float* dc_out) {
  float dc = fminf(fmaxf(dg, dmin), dmax);
  if (dc_out) *dc_out = dc;
  if (!use_precond) return 1.0f;
  const float m = dg + lam * dc;
  // the correctly rounded reciprocal: the same value as 1.0f / m, without the
  // general division's numerator handling
  return m != 0.0f ? __frcp_rn(m) : 1.0f;
}

// ---------------------------------------------------------------------------
// ARAP mesh rotation (Fig. 25 Rotate3D, read as Rz(az) Ry(ay) Rx(ax))
// ---------------------------------------------------------------------------
// Rotation R = Rz(c) Ry(b) Rx(a) applied to v, and its three angle
// derivatives applied to v (float32 kernels: RotV; float64 solver: RotVT<double>).
template <typename T>
struct RotVT {
  T rv[3];
  T g[3][3];        // g[m] = dR/dA_m v
};
using RotV = RotVT<float>;

__device__ __forceinline__ RotV rot_apply(float ax, float ay, float az, float vx, float vy, float vz) {
  float sa, ca, sb, cb, sc, cc;
  sincosf(ax, &sa, &ca);
  sincosf(ay, &sb, &cb);
  sincosf(az, &sc, &cc);
  // w = Rx v, w' = dRx v
  const float w0 = vx, w1 = ca * vy - sa * vz, w2 = sa * vy + ca * vz;
  const float wd1 = -sa * vy - ca * vz, wd2 = ca * vy - sa * vz;   // wd0 = 0
  // y = Ry w, y' (from dRy) = dRy w, ya = Ry w'
  const float y0 = cb * w0 + sb * w2, y1 = w1, y2 = -sb * w0 + cb * w2;
  const float yb0 = -sb * w0 + cb * w2, yb2 = -cb * w0 - sb * w2;     // yb1 = 0
  const float ya0 = sb * wd2, ya1 = wd1, ya2 = cb * wd2;
  RotV o;
  // R v = Rz y
  o.rv[0] = cc * y0 - sc * y1;
  o.rv[1] = sc * y0 + cc * y1;
  o.rv[2] = y2;
  // dR/dax v = Rz Ry dRx v = Rz ya
  o.g[0][0] = cc * ya0 - sc * ya1;
  o.g[0][1] = sc * ya0 + cc * ya1;
  o.g[0][2] = ya2;
  // dR/day v = Rz dRy Rx v = Rz yb
  o.g[1][0] = cc * yb0;
  o.g[1][1] = sc * yb0;
  o.g[1][2] = yb2;
  // dR/daz v = dRz Ry Rx v = dRz y
  o.g[2][0] = -sc * y0 - cc * y1;
  o.g[2][1] = cc * y0 - sc * y1;
  o.g[2][2] = 0.f;
  return o;
}

// Same as rot_apply with the angles' cos / sin given.
template <typename T>
__device__ __forceinline__ RotVT<T> rot_apply_cs(T ca, T sa, T cb, T sb, T cc, T sc, T vx, T vy, T vz) {
  const T w0 = vx, w1 = ca * vy - sa * vz, w2 = sa * vy + ca * vz;
  const T wd1 = -sa * vy - ca * vz, wd2 = ca * vy - sa * vz;
  const T y0 = cb * w0 + sb * w2, y1 = w1, y2 = -sb * w0 + cb * w2;
  const T yb0 = -sb * w0 + cb * w2, yb2 = -cb * w0 - sb * w2;
  const T ya0 = sb * wd2, ya1 = wd1, ya2 = cb * wd2;
  RotVT<T> o;
  o.rv[0] = cc * y0 - sc * y1;
  o.rv[1] = sc * y0 + cc * y1;
  o.rv[2] = y2;
  o.g[0][0] = cc * ya0 - sc * ya1;
  o.g[0][1] = sc * ya0 + cc * ya1;
  o.g[0][2] = ya2;
  o.g[1][0] = cc * yb0;
  o.g[1][1] = sc * yb0;
  o.g[1][2] = yb2;
  o.g[2][0] = -sc * y0 - cc * y1;
  o.g[2][1] = cc * y0 - sc * y1;
  o.g[2][2] = T(0);
  return o;
}

}  // namespace optgb
