// Full float64 variant of the solver (Sec. 7 "Numerical Precision": the
// solver runs in float or in double; double trades speed for stability on
// ill-conditioned problems; Fig. 14 compares both).
//
// Every quantity -- unknowns, constants, residuals, Jacobian entries,
// J^T J p, the PCG vectors, dot products and energies -- is float64.  The
// kernels compute exactly what the float32 path computes (Sec. 4.1 PCGInit /
// PCGStep split, direction update fused into applyJTJ, float64 LM decision on
// the device) for the ARAP warp (Fig. 24) and Poisson (Fig. 27) on the pixel
// grid and ARAP mesh deformation (Fig. 25) on a graph.
//
// Design.  On this part the float64 pipe is narrow: a float64 multiply-add
// issues at a small fraction of the float32 rate, while a float64 operand is
// only twice the bytes.  The float64 kernels are therefore bound by float64
// arithmetic, not by memory, and are written for the fewest float64
// operations rather than for the fewest bytes:
//  * the Jacobian entries that depend on x and are not constants -- the angle
//    columns (warp: R'(theta_i) v per residual; mesh: dR/dA_m (U_a - U_b) per
//    directed edge) -- are evaluated once per outer iteration by PCGInit and
//    read by every applyJTJ of the PCG solve (the rest of J is +-s_w);
//  * the direction update p = M^-1 r + beta p is its own streaming pass, so
//    applyJTJ reads p at the neighbours instead of re-forming it;
//  * the own and the incoming residual of a stencil pair are folded into one
//    expression (the same p differences feed both);
//  * one thread per pixel / vertex (grid-stride over a fixed grid of blocks),
//    operands straight from global memory through L1.
// Reductions are float64 throughout: per thread, per block (fixed shuffle
// tree), then across blocks in block order by the last block to arrive, so
// results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"
#include "opt_problem.h"

using namespace optgb;

namespace {

enum Kind64 : int { F64_WARP = 0, F64_POISSON = 1, F64_MESH = 2 };

// Device view of one float64 problem (passed by value to every kernel).
// Planes are dense: grid index y*W + x, graph index = vertex; n elements each.
struct P64 {
  int kind, W, H, nx;
  long long n;                  // pixels / vertices
  double s_w, s_f, w_reg, w_fit;
  int use_precond, lm;
  double* x;                    // nx planes (working copy of the unknowns)
  const double* c;              // warp U (2 planes), Poisson T (4), mesh U (3)
  const uint8_t* mask;          // grid: nonzero = excluded (warp) / fixed (Poisson); NULL = none
  const int* hslot;             // per element: handle index or -1
  const double* htgt;           // 2 (warp) or 3 (mesh) target displacements per handle
  const int* orow;              // graph: out-edges of v go to oe1[orow[v] .. orow[v+1])
  const int* oe1;
  const int* irow;              // graph: in-edges of v come from isrc[irow[v] .. irow[v+1])
  const int* isrc;
  const int* ieid;              // graph: out-edge index (into oe1) of each in-edge
  long long ne;                 // graph: directed edges
  double *d, *r, *q, *m, *dc;   // nx planes each
  double* p;                    // PCG direction (nx planes)
  double* cs;                   // cos / sin planes of the angles (warp 2, mesh 6)
  double* G;                    // angle columns of J at x: warp 8 planes of n (R'(theta) v per
                                // direction, x / y), mesh 9 planes of ne (dR/dA_m w, m-major)
  const double* pin;            // apply hook: caller direction (NULL in a solve)
  double* jtf_out;              // hook outputs (nx planes each) or NULL
  double* diag_out;
  Scalars* s;
  double* part;                 // 2 per block
  double* Ehist;
};

constexpr int kBlocksPerSM64 = 4;

// grid direction k: +x, -x, +y, -y
__device__ __forceinline__ int ddx(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
__device__ __forceinline__ int ddy(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }

#define FOR_ELEMENTS(P, i) \
  for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < (P).n; i += (long long)gridDim.x * NT)

// Block sums of a and b published to this block's slot; true in every thread
// of the last block to arrive.
__device__ __forceinline__ bool publish64(double* part, double a, double b, unsigned int* counter) {
  __shared__ int s_last;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    __stcg(&part[2 * blockIdx.x], a);
    __stcg(&part[2 * blockIdx.x + 1], b);
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return s_last != 0;
}

__device__ __forceinline__ bool elem_valid(const P64& P, long long i) { return !P.mask || P.mask[i] == 0; }

// Jacobi entry 1 / (diag + lambda clamp(diag)); 1 for a zero row or plain CG.
__device__ __forceinline__ double minv64(double dg, double lam, double dmin, double dmax, int use_precond,
                                         double* dc_out) {
  const double dcv = fmin(fmax(dg, dmin), dmax);
  *dc_out = dcv;
  if (!use_precond) return 1.0;
  const double mm = dg + lam * dcv;
  return mm != 0.0 ? 1.0 / mm : 1.0;
}

// Writes the PCGInit outputs of element i from its J^T F (g) and diag (dg).
template <int NX>
__device__ __forceinline__ double init_store(const P64& P, long long i, const double* g, const double* dg,
                                             double lam, double dmin, double dmax) {
  double rz = 0.0;
#pragma unroll
  for (int c = 0; c < NX; ++c) {
    const long long k = c * P.n + i;
    double dcv;
    const double mi = minv64(dg[c], lam, dmin, dmax, P.use_precond, &dcv);
    const double b = -g[c];
    P.r[k] = b;
    P.m[k] = mi;
    P.dc[k] = dcv;
    P.d[k] = 0.0;
    P.p[k] = mi * b;            // first direction p = z = M^-1 r
    rz += b * mi * b;
    if (P.jtf_out) P.jtf_out[k] = g[c];
    if (P.diag_out) P.diag_out[k] = dg[c];
  }
  return rz;
}

__device__ __forceinline__ void init_finish(const P64& P, double rz, double E, int k_outer) {
  if (publish64(P.part, rz, E, &P.s->counter)) {
    gather_partials(P.part, 0, gridDim.x, &P.s->counter, rz, E);
    if (threadIdx.x == 0) {
      Scalars* s = P.s;
      s->rz = rz;
      s->E = E;
      if (P.Ehist && k_outer >= 0) P.Ehist[k_outer] = E;
      s->beta_d = 0.0;
      s->pcg_active = (rz != 0.0) && isfinite(rz);
      if (!isfinite(rz) || !isfinite(E)) s->nonfinite = 1;
    }
  }
}

__device__ __forceinline__ void apply_finish(const P64& P, double pq) {
  if (publish64(P.part, pq, 0.0, &P.s->counter)) {
    double unused;
    gather_partials(P.part, 0, gridDim.x, &P.s->counter, pq, unused);
    if (threadIdx.x == 0) {
      Scalars* s = P.s;
      s->pq = pq;
      if (pq > 0.0 && isfinite(pq)) {
        s->alpha_d = s->rz / pq;
      } else {
        s->alpha_d = 0.0;
        s->pcg_active = 0;
        if (!isfinite(pq)) s->nonfinite = 1;
      }
    }
  }
}

__device__ __forceinline__ void energy_finish(const P64& P, double e0, double e1, int mode, int hist_idx) {
  if (publish64(P.part, e0, e1, &P.s->counter)) {
    gather_partials(P.part, 0, gridDim.x, &P.s->counter, e0, e1);
    if (threadIdx.x == 0) {
      Scalars* s = P.s;
      if (mode == 0) {
        s->E = e0;
        const int k = hist_idx >= 0 ? hist_idx : (hist_idx == -1 ? s->outer_done : -1);
        if (P.Ehist && k >= 0) P.Ehist[k] = e0;
        if (!isfinite(e0)) s->nonfinite = 1;
      } else {
        s->E_trial = e0;
        s->model = e1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// shared kernels
// ---------------------------------------------------------------------------
__global__ void k64_reset(Scalars* s, double lambda0) { scalars_reset(s, lambda0); }

__global__ void k64_force_active(Scalars* s) {
  s->pcg_active = 1;
  s->done = 0;
}

__global__ void k64_lm_decide(Scalars* s, double eta, double lmin, double lmax, double rel_tol) {
  lm_decide(s, eta, lmin, lmax, rel_tol);
}

// cos / sin of the rotation angles at x (warp: theta; mesh: ax, ay, az),
// once per outer iteration (Sec. 4.2: evalJ's values depend only on x).
__global__ void __launch_bounds__(NT) k64_rot(P64 P) {
  const int na = P.kind == F64_WARP ? 1 : 3;
  const int a0 = P.kind == F64_WARP ? 2 : 3;
  FOR_ELEMENTS(P, i) {
    for (int a = 0; a < na; ++a) {
      double sn, cn;
      sincos(P.x[(a0 + a) * P.n + i], &sn, &cn);
      P.cs[(2 * a) * P.n + i] = cn;
      P.cs[(2 * a + 1) * P.n + i] = sn;
    }
  }
}

// Direction update (Sec. 4.1 PCGStep): p = z + beta p, z = M^-1 r (every
// PCG iteration after the first; PCGInit writes the first direction).
template <int NX>
__global__ void __launch_bounds__(NT) k64_direction(P64 P) {
  const Scalars* s = P.s;
  if (s->done || !s->pcg_active) return;
  const double beta = s->beta_d;
  double* __restrict__ pp = P.p;
  const double* __restrict__ mm = P.m;
  const double* __restrict__ rr = P.r;
  FOR_ELEMENTS(P, i) {
    double pv[NX], mv[NX], rv[NX];   // every load before any store
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      pv[c] = pp[c * P.n + i];
      mv[c] = mm[c * P.n + i];
      rv[c] = rr[c * P.n + i];
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) pp[c * P.n + i] = fma(beta, pv[c], mv[c] * rv[c]);
  }
}

// PCG vector update (Sec. 4.1 PCGStep): delta += alpha p, r -= alpha q,
// z = M^-1 r, r.z -> beta = r.z / r.z_old.
template <int NX>
__global__ void __launch_bounds__(NT) k64_update(P64 P) {
  Scalars* s = P.s;
  if (s->done || !s->pcg_active) return;
  const double alpha = s->alpha_d;
  const double* __restrict__ pn = P.p;
  const double* __restrict__ qq = P.q;
  const double* __restrict__ mm = P.m;
  double* __restrict__ dd = P.d;
  double* __restrict__ rr = P.r;
  double rz = 0.0;
  FOR_ELEMENTS(P, i) {
    double pv[NX], qv[NX], mv[NX], dv[NX], rv[NX];   // every load before any store
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      const long long k = c * P.n + i;
      pv[c] = pn[k];
      qv[c] = qq[k];
      mv[c] = mm[k];
      dv[c] = dd[k];
      rv[c] = rr[k];
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      const long long k = c * P.n + i;
      dd[k] = fma(alpha, pv[c], dv[c]);
      const double r2 = fma(-alpha, qv[c], rv[c]);
      rr[k] = r2;
      rz += r2 * mv[c] * r2;
    }
  }
  if (publish64(P.part, rz, 0.0, &s->counter)) {
    double unused;
    gather_partials(P.part, 0, gridDim.x, &s->counter, rz, unused);
    if (threadIdx.x == 0) {
      s->beta_d = rz / s->rz;
      s->rz = rz;
      s->pcg_iters += 1;
      if (rz == 0.0 || !isfinite(rz)) s->pcg_active = 0;
      if (!isfinite(rz)) s->nonfinite = 1;
    }
  }
}

// x += delta (cond 0: unless the solve is done; cond 1: only if LM accepted).
__global__ void __launch_bounds__(NT) k64_step(P64 P, int cond) {
  const Scalars* s = P.s;
  if (cond ? !s->accept : s->done) return;
  FOR_ELEMENTS(P, i) {
    for (int c = 0; c < P.nx; ++c) P.x[c * P.n + i] += P.d[c * P.n + i];
  }
}

// ---------------------------------------------------------------------------
// ARAP image warping (Fig. 24): unknowns dx, dy, theta; O = U + (dx, dy).
// Residual (k, d) for valid k, k+d: s_w ((O_k - O_{k+d}) - R(theta_k) v),
// v = U_k - U_{k+d}; handle h: s_f (O_h - C_h) = s_f ((dx, dy)_h - target).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k64_warp_init(P64 P, int k_outer, double dmin, double dmax) {
  Scalars* s = P.s;
  if (s->done) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const long long n = P.n;
  const double sw = P.s_w, w = P.w_reg;
  double rz = 0.0, E = 0.0;
  FOR_ELEMENTS(P, i) {
    double g[3] = {0.0, 0.0, 0.0}, dg[3] = {0.0, 0.0, 0.0};
    if (elem_valid(P, i)) {
      const int gx = (int)(i % P.W), gy = (int)(i / P.W);
      const double xi = P.x[i], yi = P.x[n + i];
      const double ci = P.cs[i], si = P.cs[n + i];
      const double uxi = P.c[i], uyi = P.c[n + i];
      for (int k = 0; k < 4; ++k) {
        P.G[(2 * k) * n + i] = 0.0;
        P.G[(2 * k + 1) * n + i] = 0.0;
        const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
        if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
        const long long j = (long long)ny_ * P.W + nx_;
        if (!elem_valid(P, j)) continue;
        const double vx = uxi - P.c[j], vy = uyi - P.c[n + j];
        const double xj = P.x[j], yj = P.x[n + j];
        // own residual (i, d)
        const double fx = sw * ((xi - xj) + vx - (ci * vx - si * vy));
        const double fy = sw * ((yi - yj) + vy - (si * vx + ci * vy));
        const double rpx = -si * vx - ci * vy, rpy = ci * vx - si * vy;   // R'(theta_i) v
        P.G[(2 * k) * n + i] = rpx;
        P.G[(2 * k + 1) * n + i] = rpy;
        E += fx * fx + fy * fy;
        g[0] += sw * fx;
        g[1] += sw * fy;
        g[2] -= sw * (rpx * fx + rpy * fy);
        dg[0] += w;
        dg[1] += w;
        dg[2] += w * (rpx * rpx + rpy * rpy);
        // incoming residual (j, -d): d/dO_i = -s_w I
        const double cj = P.cs[j], sj = P.cs[n + j];
        const double wx = -vx, wy = -vy;
        const double hx = sw * ((xj - xi) + wx - (cj * wx - sj * wy));
        const double hy = sw * ((yj - yi) + wy - (sj * wx + cj * wy));
        g[0] -= sw * hx;
        g[1] -= sw * hy;
        dg[0] += w;
        dg[1] += w;
      }
      const int h = P.hslot[i];
      if (h >= 0) {
        const double fx = P.s_f * (xi - P.htgt[2 * h]), fy = P.s_f * (yi - P.htgt[2 * h + 1]);
        E += fx * fx + fy * fy;
        g[0] += P.s_f * fx;
        g[1] += P.s_f * fy;
        dg[0] += P.w_fit;
        dg[1] += P.w_fit;
      }
    }
    rz += init_store<3>(P, i, g, dg, lam, dmin, dmax);
  }
  init_finish(P, rz, E, k_outer);
}

// q = (J^T J + lambda D) p with the angle columns of J from PCGInit; p.q ->
// alpha.  Per stencil pair (i, j = i + d), both residuals exist together
// (both pixels valid); with dp = p_i - p_j (x, y), a = dp - R'_i v pt_i the
// own row's J p / s_w and b = -dp - R'_j (-v) pt_j the incoming one's:
//   q_O += w (a - b) = w (a + dp + R'_j(-v) pt_j),   q_t -= w R'_i v . a.
__global__ void __launch_bounds__(NT) k64_warp_apply(P64 P) {
  Scalars* s = P.s;
  if (s->done || !s->pcg_active) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const double* __restrict__ pp = P.pin ? P.pin : P.p;
  const long long n = P.n;
  const double w = P.w_reg;
  double pq = 0.0;
  FOR_ELEMENTS(P, i) {
    // rows without residuals (excluded pixels) carry only the damping term
    const double pxi = pp[i], pyi = pp[n + i], pti = pp[2 * n + i];
    double ax_ = 0.0, ay_ = 0.0, at_ = 0.0;
    if (elem_valid(P, i)) {
      const int gx = (int)(i % P.W), gy = (int)(i / P.W);
      for (int k = 0; k < 4; ++k) {
        const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
        if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
        const long long j = (long long)ny_ * P.W + nx_;
        if (!elem_valid(P, j)) continue;
        const int ko = k ^ 1;                                   // the opposite direction, seen from j
        const double rpx = P.G[(2 * k) * n + i], rpy = P.G[(2 * k + 1) * n + i];
        const double qpx = P.G[(2 * ko) * n + j], qpy = P.G[(2 * ko + 1) * n + j];
        const double ptj = pp[2 * n + j];
        const double dx = pxi - pp[j], dy = pyi - pp[n + j];
        const double ax = fma(-rpx, pti, dx), ay = fma(-rpy, pti, dy);
        at_ = fma(rpx, ax, fma(rpy, ay, at_));
        ax_ += fma(qpx, ptj, ax + dx);
        ay_ += fma(qpy, ptj, ay + dy);
      }
    }
    double qx = w * ax_, qy = w * ay_, qt = -w * at_;
    if (P.hslot[i] >= 0) {
      qx = fma(P.w_fit, pxi, qx);
      qy = fma(P.w_fit, pyi, qy);
    }
    if (lam != 0.0) {
      qx += lam * P.dc[i] * pxi;
      qy += lam * P.dc[n + i] * pyi;
      qt += lam * P.dc[2 * n + i] * pti;
    }
    P.q[i] = qx;
    P.q[n + i] = qy;
    P.q[2 * n + i] = qt;
    pq += pxi * qx + pyi * qy + pti * qt;
  }
  apply_finish(P, pq);
}

// E(x) (mode 0) or E(x + delta) and |F(x) + J(x) delta|^2 (mode 1).
__global__ void __launch_bounds__(NT) k64_warp_energy(P64 P, int mode, int hist_idx) {
  Scalars* s = P.s;
  if (mode == 1 && s->done) return;
  const long long n = P.n;
  const double sw = P.s_w;
  double e0 = 0.0, e1 = 0.0;
  FOR_ELEMENTS(P, i) {
    if (!elem_valid(P, i)) continue;
    const int gx = (int)(i % P.W), gy = (int)(i / P.W);
    const double xi = P.x[i], yi = P.x[n + i], ti = P.x[2 * n + i];
    double si, ci, s2 = 0.0, c2 = 0.0;
    sincos(ti, &si, &ci);
    double exi = 0.0, eyi = 0.0, eti = 0.0;
    if (mode == 1) {
      exi = P.d[i];
      eyi = P.d[n + i];
      eti = P.d[2 * n + i];
      sincos(ti + eti, &s2, &c2);
    }
    const double uxi = P.c[i], uyi = P.c[n + i];
    for (int k = 0; k < 4; ++k) {
      const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
      if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
      const long long j = (long long)ny_ * P.W + nx_;
      if (!elem_valid(P, j)) continue;
      const double vx = uxi - P.c[j], vy = uyi - P.c[n + j];
      const double ddx_ = xi - P.x[j], ddy_ = yi - P.x[n + j];
      const double fx = sw * (ddx_ + vx - (ci * vx - si * vy));
      const double fy = sw * (ddy_ + vy - (si * vx + ci * vy));
      if (mode == 0) {
        e0 += fx * fx + fy * fy;
      } else {
        const double edx = exi - P.d[j], edy = eyi - P.d[n + j];
        const double tx = sw * ((ddx_ + edx) + vx - (c2 * vx - s2 * vy));
        const double ty = sw * ((ddy_ + edy) + vy - (s2 * vx + c2 * vy));
        e0 += tx * tx + ty * ty;
        const double lx = fx + sw * (edx - (-si * vx - ci * vy) * eti);
        const double ly = fy + sw * (edy - (ci * vx - si * vy) * eti);
        e1 += lx * lx + ly * ly;
      }
    }
    const int h = P.hslot[i];
    if (h >= 0) {
      const double fx = P.s_f * (xi + exi - P.htgt[2 * h]), fy = P.s_f * (yi + eyi - P.htgt[2 * h + 1]);
      e0 += fx * fx + fy * fy;   // linear in delta: trial == model
      e1 += fx * fx + fy * fy;
    }
  }
  energy_finish(P, e0, e1, mode, hist_idx);
}

// ---------------------------------------------------------------------------
// Poisson image editing (Fig. 27), 4 channels.  Free pixel k (mask 0) and
// neighbour k+d in the image: residual (X_k - X_{k+d}) - (T_k - T_{k+d});
// fixed pixels' X are constants.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k64_poisson_init(P64 P, int k_outer, double dmin, double dmax) {
  Scalars* s = P.s;
  if (s->done) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const long long n = P.n;
  double rz = 0.0, E = 0.0;
  FOR_ELEMENTS(P, i) {
    double g[4] = {0.0, 0.0, 0.0, 0.0}, dg[4] = {0.0, 0.0, 0.0, 0.0};
    if (elem_valid(P, i)) {
      const int gx = (int)(i % P.W), gy = (int)(i / P.W);
      double cnt = 0.0;
      for (int k = 0; k < 4; ++k) {
        const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
        if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
        const long long j = (long long)ny_ * P.W + nx_;
        const bool fj = elem_valid(P, j);
        cnt += fj ? 2.0 : 1.0;
        for (int c = 0; c < 4; ++c) {
          const long long a = c * n;
          const double f = (P.x[a + i] - P.x[a + j]) - (P.c[a + i] - P.c[a + j]);
          E += f * f;
          g[c] += f;
          if (fj) g[c] += f;   // incoming residual (j, -d) = -f, d/dX_i = -1
        }
      }
      for (int c = 0; c < 4; ++c) dg[c] = cnt;
    }
    rz += init_store<4>(P, i, g, dg, lam, dmin, dmax);
  }
  init_finish(P, rz, E, k_outer);
}

__global__ void __launch_bounds__(NT) k64_poisson_apply(P64 P) {
  Scalars* s = P.s;
  if (s->done || !s->pcg_active) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const double* __restrict__ pp = P.pin ? P.pin : P.p;
  const long long n = P.n;
  double pq = 0.0;
  FOR_ELEMENTS(P, i) {
    // fixed pixels carry only the damping term (their p is 0 in a solve)
    double pv[4], qv[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 4; ++c) pv[c] = pp[c * n + i];
    if (elem_valid(P, i)) {
      const int gx = (int)(i % P.W), gy = (int)(i / P.W);
      for (int k = 0; k < 4; ++k) {
        const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
        if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
        const long long j = (long long)ny_ * P.W + nx_;
        // own residual: J p = p_i - p_j (p_j = 0 on a fixed pixel); the
        // incoming one of a free neighbour adds the same again
        const bool fj = elem_valid(P, j);
        const double f = fj ? 2.0 : 1.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) qv[c] = fma(f, pv[c] - (fj ? pp[c * n + j] : 0.0), qv[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (lam != 0.0) qv[c] += lam * P.dc[c * n + i] * pv[c];
      P.q[c * n + i] = qv[c];
      pq += pv[c] * qv[c];
    }
  }
  apply_finish(P, pq);
}

__global__ void __launch_bounds__(NT) k64_poisson_energy(P64 P, int mode, int hist_idx) {
  Scalars* s = P.s;
  if (mode == 1 && s->done) return;
  const long long n = P.n;
  double e0 = 0.0, e1 = 0.0;
  FOR_ELEMENTS(P, i) {
    if (!elem_valid(P, i)) continue;
    const int gx = (int)(i % P.W), gy = (int)(i / P.W);
    for (int k = 0; k < 4; ++k) {
      const int nx_ = gx + ddx(k), ny_ = gy + ddy(k);
      if (nx_ < 0 || nx_ >= P.W || ny_ < 0 || ny_ >= P.H) continue;
      const long long j = (long long)ny_ * P.W + nx_;
      for (int c = 0; c < 4; ++c) {
        const long long a = c * n;
        const double f = (P.x[a + i] - P.x[a + j]) - (P.c[a + i] - P.c[a + j]);
        if (mode == 0) {
          e0 += f * f;
        } else {
          // delta is 0 on fixed pixels; J is constant, so trial and model agree
          const double t = f + (P.d[a + i] - P.d[a + j]);
          e0 += t * t;
          e1 += t * t;
        }
      }
    }
  }
  energy_finish(P, e0, e1, mode, hist_idx);
}

// ---------------------------------------------------------------------------
// ARAP mesh deformation (Fig. 25): unknowns displacement d (3) and Euler
// angles A (3) per vertex; residual of edge (a, b):
// s_w ((O_a - O_b) - Rz Ry Rx(A_a) (U_a - U_b)); handle: s_f (O_h - C_h).
// Vertex-centric gather: a vertex sums its out-edges' rows (own residuals)
// and its in-edges' rows (far-end residuals), so no atomics are needed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ RotVT<double> rot_at(const P64& P, long long v, double wx, double wy, double wz) {
  const long long n = P.n;
  return rot_apply_cs<double>(P.cs[v], P.cs[n + v], P.cs[2 * n + v], P.cs[3 * n + v], P.cs[4 * n + v],
                              P.cs[5 * n + v], wx, wy, wz);
}

__global__ void __launch_bounds__(NT) k64_mesh_init(P64 P, int k_outer, double dmin, double dmax) {
  Scalars* s = P.s;
  if (s->done) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const long long n = P.n;
  const double sw = P.s_w, w = P.w_reg;
  double rz = 0.0, E = 0.0;
  FOR_ELEMENTS(P, v) {
    double g[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, dg[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double xv[3] = {P.x[v], P.x[n + v], P.x[2 * n + v]};
    const double uv[3] = {P.c[v], P.c[n + v], P.c[2 * n + v]};
    for (int e = P.orow[v]; e < P.orow[v + 1]; ++e) {
      const int b = P.oe1[e];
      const double wv[3] = {uv[0] - P.c[b], uv[1] - P.c[n + b], uv[2] - P.c[2 * n + b]};
      const RotVT<double> R = rot_at(P, v, wv[0], wv[1], wv[2]);
      for (int m = 0; m < 3; ++m)
        for (int c = 0; c < 3; ++c) P.G[(3 * m + c) * P.ne + e] = R.g[m][c];
      double f[3];
      for (int c = 0; c < 3; ++c) f[c] = sw * ((xv[c] - P.x[c * n + b]) + wv[c] - R.rv[c]);
      E += f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
      for (int c = 0; c < 3; ++c) {
        g[c] += sw * f[c];
        dg[c] += w;
      }
      for (int m = 0; m < 3; ++m) {
        g[3 + m] -= sw * (R.g[m][0] * f[0] + R.g[m][1] * f[1] + R.g[m][2] * f[2]);
        dg[3 + m] += w * (R.g[m][0] * R.g[m][0] + R.g[m][1] * R.g[m][1] + R.g[m][2] * R.g[m][2]);
      }
    }
    for (int e = P.irow[v]; e < P.irow[v + 1]; ++e) {
      const int a = P.isrc[e];
      const double wv[3] = {P.c[a] - uv[0], P.c[n + a] - uv[1], P.c[2 * n + a] - uv[2]};
      const RotVT<double> R = rot_at(P, a, wv[0], wv[1], wv[2]);
      for (int c = 0; c < 3; ++c) {
        const double f = sw * ((P.x[c * n + a] - xv[c]) + wv[c] - R.rv[c]);
        g[c] -= sw * f;
        dg[c] += w;
      }
    }
    const int h = P.hslot[v];
    if (h >= 0) {
      for (int c = 0; c < 3; ++c) {
        const double f = P.s_f * (xv[c] - P.htgt[3 * h + c]);
        E += f * f;
        g[c] += P.s_f * f;
        dg[c] += P.w_fit;
      }
    }
    rz += init_store<6>(P, v, g, dg, lam, dmin, dmax);
  }
  init_finish(P, rz, E, k_outer);
}

// q = (J^T J + lambda D) p with every edge's angle columns g_m = dR/dA_m w
// (w = U_a - U_b) from PCGInit: J_e p / s_w = (pd_a - pd_b) - sum_m g_m pA_m(a);
// own edges add w J_e p / s_w to q_d and -w g_m . (J_e p / s_w) to q_A, in-edges
// subtract w J_e p / s_w from q_d.
__global__ void __launch_bounds__(NT) k64_mesh_apply(P64 P) {
  Scalars* s = P.s;
  if (s->done || !s->pcg_active) return;
  const double lam = P.lm ? s->lambda : 0.0;
  const double* __restrict__ pp = P.pin ? P.pin : P.p;
  const long long n = P.n, ne = P.ne;
  const double w = P.w_reg;
  double pq = 0.0;
  FOR_ELEMENTS(P, v) {
    double pv[6], qd[3] = {0.0, 0.0, 0.0}, qa[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 6; ++c) pv[c] = pp[c * n + v];
    for (int e = P.orow[v]; e < P.orow[v + 1]; ++e) {
      const int b = P.oe1[e];
      double g[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = P.G[k * ne + e];
      double jp[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double t = fma(g[c], pv[3], fma(g[3 + c], pv[4], g[6 + c] * pv[5]));
        jp[c] = (pv[c] - pp[c * n + b]) - t;
        qd[c] += jp[c];
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) qa[m] = fma(g[3 * m], jp[0], fma(g[3 * m + 1], jp[1], fma(g[3 * m + 2], jp[2], qa[m])));
    }
    for (int k = P.irow[v]; k < P.irow[v + 1]; ++k) {
      const int a = P.isrc[k], e = P.ieid[k];
      const double pa3 = pp[3 * n + a], pa4 = pp[4 * n + a], pa5 = pp[5 * n + a];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double t = fma(P.G[c * ne + e], pa3, fma(P.G[(3 + c) * ne + e], pa4, P.G[(6 + c) * ne + e] * pa5));
        qd[c] -= (pp[c * n + a] - pv[c]) - t;
      }
    }
    double qv[6] = {w * qd[0], w * qd[1], w * qd[2], -w * qa[0], -w * qa[1], -w * qa[2]};
    if (P.hslot[v] >= 0)
#pragma unroll
      for (int c = 0; c < 3; ++c) qv[c] = fma(P.w_fit, pv[c], qv[c]);
    if (lam != 0.0)
#pragma unroll
      for (int c = 0; c < 6; ++c) qv[c] += lam * P.dc[c * n + v] * pv[c];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      P.q[c * n + v] = qv[c];
      pq += pv[c] * qv[c];
    }
  }
  apply_finish(P, pq);
}

__global__ void __launch_bounds__(NT) k64_mesh_energy(P64 P, int mode, int hist_idx) {
  Scalars* s = P.s;
  if (mode == 1 && s->done) return;
  const long long n = P.n;
  const double sw = P.s_w;
  double e0 = 0.0, e1 = 0.0;
  FOR_ELEMENTS(P, v) {
    double cs[6], cs2[6], ev[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) sincos(P.x[(3 + a) * n + v], &cs[2 * a + 1], &cs[2 * a]);
    if (mode == 1) {
      for (int c = 0; c < 6; ++c) ev[c] = P.d[c * n + v];
      for (int a = 0; a < 3; ++a) sincos(P.x[(3 + a) * n + v] + ev[3 + a], &cs2[2 * a + 1], &cs2[2 * a]);
    }
    const double xv[3] = {P.x[v], P.x[n + v], P.x[2 * n + v]};
    const double uv[3] = {P.c[v], P.c[n + v], P.c[2 * n + v]};
    for (int e = P.orow[v]; e < P.orow[v + 1]; ++e) {
      const int b = P.oe1[e];
      const double wv[3] = {uv[0] - P.c[b], uv[1] - P.c[n + b], uv[2] - P.c[2 * n + b]};
      const RotVT<double> R =
          rot_apply_cs<double>(cs[0], cs[1], cs[2], cs[3], cs[4], cs[5], wv[0], wv[1], wv[2]);
      double f[3];
      for (int c = 0; c < 3; ++c) f[c] = sw * ((xv[c] - P.x[c * n + b]) + wv[c] - R.rv[c]);
      if (mode == 0) {
        e0 += f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
        continue;
      }
      const RotVT<double> R2 =
          rot_apply_cs<double>(cs2[0], cs2[1], cs2[2], cs2[3], cs2[4], cs2[5], wv[0], wv[1], wv[2]);
      for (int c = 0; c < 3; ++c) {
        const double ed = ev[c] - P.d[c * n + b];
        const double t = sw * ((xv[c] - P.x[c * n + b] + ed) + wv[c] - R2.rv[c]);
        const double l = f[c] + sw * (ed - (R.g[0][c] * ev[3] + R.g[1][c] * ev[4] + R.g[2][c] * ev[5]));
        e0 += t * t;
        e1 += l * l;
      }
    }
    const int h = P.hslot[v];
    if (h >= 0) {
      for (int c = 0; c < 3; ++c) {
        const double f = P.s_f * (xv[c] + ev[c] - P.htgt[3 * h + c]);
        e0 += f * f;
        e1 += f * f;
      }
    }
  }
  energy_finish(P, e0, e1, mode, hist_idx);
}

// Float64 multiply-add throughput probe: 8 independent dependency chains per
// thread, enough blocks to fill every SM; the result is consumed so the
// chains are not removed.
__global__ void __launch_bounds__(NT) k64_fma_probe(double* out, int iters, double a, double b) {
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  if (t == -1.0) out[blockIdx.x] = t;   // never true for the probe's a, b
}

}  // namespace

// =============================================================================
// host side
// =============================================================================
struct opt_problem_f64 {
  int kind = 0, nx = 0, sms = 148, nblk = 1;
  P64 hp{};
  double* user_x[6] = {};
  std::vector<void*> allocs;
  Scalars* d_s = nullptr;
  double* d_Ehist = nullptr;
  int Ehist_cap = 0;
  double* d_pin = nullptr;      // apply hook: caller p copied here (nx planes)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> gkey;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  ~opt_problem_f64() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (void* a : allocs) cudaFree(a);
  }
};

namespace {

opt_status fail64(cudaError_t e, const char* what) { return optgb::cuda_fail(e, what); }

#define CK64(call)                                      \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return fail64(e_, #call);    \
  } while (0)
#define CKS64(call)                    \
  do {                                 \
    opt_status s_ = (call);            \
    if (s_ != OPT_OK) return s_;       \
  } while (0)

template <typename T>
opt_status alloc64(opt_problem_f64* pb, T** out, size_t count) {
  void* ptr = nullptr;
  CK64(cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T)));
  pb->allocs.push_back(ptr);
  *out = static_cast<T*>(ptr);
  return OPT_OK;
}

template <typename T>
opt_status upload64(opt_problem_f64* pb, T** out, const std::vector<T>& h) {
  CKS64(alloc64(pb, out, h.size()));
  if (!h.empty()) CK64(cudaMemcpy(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return OPT_OK;
}

template <typename T>
opt_status download64(std::vector<T>& h, const T* d, size_t count) {
  h.resize(count);
  if (count) CK64(cudaMemcpy(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost));
  return OPT_OK;
}

bool all_finite(const std::vector<double>& v) {
  for (double a : v)
    if (!std::isfinite(a)) return false;
  return true;
}

// Allocates scratch and fills the common descriptor fields.
opt_status plan_common(opt_problem_f64* pb, const std::vector<double>& consts, const std::vector<int>& hslot,
                       const std::vector<double>& htgt, double w_reg, double w_fit) {
  P64& P = pb->hp;
  const size_t n = (size_t)P.n;
  int dev = 0;
  CK64(cudaGetDevice(&dev));
  CK64(cudaDeviceGetAttribute(&pb->sms, cudaDevAttrMultiProcessorCount, dev));
  const long long full = (P.n + NT - 1) / NT;
  pb->nblk = (int)std::max<long long>(1, std::min<long long>(full, (long long)kBlocksPerSM64 * pb->sms));
  P.w_reg = w_reg;
  P.w_fit = w_fit;
  P.s_w = std::sqrt(w_reg);
  P.s_f = std::sqrt(w_fit);
  P.use_precond = 1;
  double* c = nullptr;
  CKS64(upload64(pb, &c, consts));
  P.c = c;
  int* hs = nullptr;
  CKS64(upload64(pb, &hs, hslot));
  P.hslot = hs;
  double* ht = nullptr;
  CKS64(upload64(pb, &ht, htgt));
  P.htgt = ht;
  const int ncs = P.kind == F64_WARP ? 2 : (P.kind == F64_MESH ? 6 : 0);
  CKS64(alloc64(pb, &P.x, n * P.nx));
  CKS64(alloc64(pb, &P.d, n * P.nx));
  CKS64(alloc64(pb, &P.r, n * P.nx));
  CKS64(alloc64(pb, &P.q, n * P.nx));
  CKS64(alloc64(pb, &P.m, n * P.nx));
  CKS64(alloc64(pb, &P.dc, n * P.nx));
  CKS64(alloc64(pb, &P.p, n * P.nx));
  CKS64(alloc64(pb, &pb->d_pin, n * P.nx));
  if (ncs) CKS64(alloc64(pb, &P.cs, n * ncs));
  CKS64(alloc64(pb, &P.part, 2 * (size_t)pb->nblk));
  CKS64(alloc64(pb, &pb->d_s, 1));
  CK64(cudaMemset(pb->d_s, 0, sizeof(Scalars)));
  CK64(cudaMemset(P.p, 0, n * P.nx * sizeof(double)));
  P.s = pb->d_s;
  CK64(cudaStreamCreateWithFlags(&pb->cap_stream, cudaStreamNonBlocking));
  CK64(cudaEventCreate(&pb->ev0));
  CK64(cudaEventCreate(&pb->ev1));
  return OPT_OK;
}

// Handle slots: OPT_ERR_INVALID_ARG on an index outside [0, n) or a repeat.
opt_status handle_slots(const int32_t* d_idx, int nh, long long n, std::vector<int>& hslot, std::vector<int>& hidx) {
  hslot.assign((size_t)n, -1);
  hidx.clear();
  if (nh < 0) return OPT_ERR_INVALID_ARG;
  if (nh == 0) return OPT_OK;
  if (!d_idx) return OPT_ERR_INVALID_ARG;
  CKS64(download64(hidx, d_idx, (size_t)nh));
  for (int h = 0; h < nh; ++h) {
    const int i = hidx[h];
    if (i < 0 || i >= n || hslot[(size_t)i] != -1) return OPT_ERR_INVALID_ARG;
    hslot[(size_t)i] = h;
  }
  return OPT_OK;
}

// Launch set of one phase.
void k_rot(opt_problem_f64* pb, cudaStream_t st) {
  if (pb->kind != F64_POISSON) k64_rot<<<pb->nblk, NT, 0, st>>>(pb->hp);
}
void k_init(opt_problem_f64* pb, const P64& P, cudaStream_t st, int k, double dmin, double dmax) {
  if (pb->kind == F64_WARP) k64_warp_init<<<pb->nblk, NT, 0, st>>>(P, k, dmin, dmax);
  else if (pb->kind == F64_POISSON) k64_poisson_init<<<pb->nblk, NT, 0, st>>>(P, k, dmin, dmax);
  else k64_mesh_init<<<pb->nblk, NT, 0, st>>>(P, k, dmin, dmax);
}
// applyJTJ of PCG iteration i: the direction update (from the second
// iteration on; PCGInit writes the first direction), then q = A p
void k_apply(opt_problem_f64* pb, const P64& P, cudaStream_t st, int i) {
  if (i > 0 && !P.pin) {
    if (pb->kind == F64_WARP) k64_direction<3><<<pb->nblk, NT, 0, st>>>(P);
    else if (pb->kind == F64_POISSON) k64_direction<4><<<pb->nblk, NT, 0, st>>>(P);
    else k64_direction<6><<<pb->nblk, NT, 0, st>>>(P);
  }
  if (pb->kind == F64_WARP) k64_warp_apply<<<pb->nblk, NT, 0, st>>>(P);
  else if (pb->kind == F64_POISSON) k64_poisson_apply<<<pb->nblk, NT, 0, st>>>(P);
  else k64_mesh_apply<<<pb->nblk, NT, 0, st>>>(P);
}
void k_update(opt_problem_f64* pb, const P64& P, cudaStream_t st) {
  if (pb->kind == F64_WARP) k64_update<3><<<pb->nblk, NT, 0, st>>>(P);
  else if (pb->kind == F64_POISSON) k64_update<4><<<pb->nblk, NT, 0, st>>>(P);
  else k64_update<6><<<pb->nblk, NT, 0, st>>>(P);
}
void k_energy(opt_problem_f64* pb, const P64& P, cudaStream_t st, int mode, int hist) {
  if (pb->kind == F64_WARP) k64_warp_energy<<<pb->nblk, NT, 0, st>>>(P, mode, hist);
  else if (pb->kind == F64_POISSON) k64_poisson_energy<<<pb->nblk, NT, 0, st>>>(P, mode, hist);
  else k64_mesh_energy<<<pb->nblk, NT, 0, st>>>(P, mode, hist);
}

opt_status copy_x(opt_problem_f64* pb, bool in, cudaStream_t st) {
  const size_t bytes = (size_t)pb->hp.n * sizeof(double);
  for (int c = 0; c < pb->nx; ++c) {
    double* dev = pb->hp.x + (size_t)c * pb->hp.n;
    if (in) CK64(cudaMemcpyAsync(dev, pb->user_x[c], bytes, cudaMemcpyDeviceToDevice, st));
    else CK64(cudaMemcpyAsync(pb->user_x[c], dev, bytes, cudaMemcpyDeviceToDevice, st));
  }
  return OPT_OK;
}

opt_status check_params64(const opt_solve_params& p, bool lm) {
  if (p.outer < 1 || p.inner < 0 || p.outer > (1 << 20) || p.inner > (1 << 20)) return OPT_ERR_INVALID_ARG;
  if (p.use_precond != 0 && p.use_precond != 1) return OPT_ERR_INVALID_ARG;
  if (p.materialized != 0) return OPT_ERR_INVALID_ARG;   // matrix-free only
  if (lm) {
    if (!(p.lambda0 >= 0.0) || !std::isfinite(p.lambda0)) return OPT_ERR_INVALID_ARG;
    if (!(p.lambda_min >= 0.0) || !(p.lambda_min <= p.lambda_max)) return OPT_ERR_INVALID_ARG;
    if (!(p.diag_min >= 0.0) || !(p.diag_min <= p.diag_max)) return OPT_ERR_INVALID_ARG;
    if (!std::isfinite(p.eta) || !(p.rel_tol >= 0.0)) return OPT_ERR_INVALID_ARG;
  }
  return OPT_OK;
}

opt_status enqueue_solve64(opt_problem_f64* pb, const opt_solve_params& p, bool lm, cudaStream_t st) {
  P64 P = pb->hp;
  P.lm = lm ? 1 : 0;
  P.use_precond = p.use_precond;
  P.Ehist = pb->d_Ehist;
  pb->hp = P;
  CKS64(copy_x(pb, true, st));
  k64_reset<<<1, 1, 0, st>>>(pb->d_s, lm ? p.lambda0 : 0.0);
  for (int k = 0; k < p.outer; ++k) {
    k_rot(pb, st);
    k_init(pb, P, st, k, p.diag_min, p.diag_max);
    for (int i = 0; i < p.inner; ++i) {
      k_apply(pb, P, st, i);
      k_update(pb, P, st);
    }
    if (!lm) {
      k64_step<<<pb->nblk, NT, 0, st>>>(P, 0);
    } else {
      k_energy(pb, P, st, 1, -2);
      k64_lm_decide<<<1, 1, 0, st>>>(pb->d_s, p.eta, p.lambda_min, p.lambda_max, p.rel_tol);
      k64_step<<<pb->nblk, NT, 0, st>>>(P, 1);
    }
  }
  k_energy(pb, P, st, 0, lm ? -1 : p.outer);
  CKS64(copy_x(pb, false, st));
  CK64(cudaGetLastError());
  return OPT_OK;
}

opt_status run_solve64(opt_problem_f64* pb, const opt_solve_params* prm_in, opt_report* rep, bool lm) {
  if (!pb) return OPT_ERR_INVALID_ARG;
  opt_solve_params p;
  if (prm_in) p = *prm_in;
  else opt_solve_params_default(&p);
  CKS64(check_params64(p, lm));
  cudaStream_t st = (cudaStream_t)p.stream;
  CK64(cudaStreamSynchronize(st));
  if (pb->Ehist_cap < p.outer + 1) {
    if (pb->gexec) {
      cudaGraphExecDestroy(pb->gexec);
      pb->gexec = nullptr;
      pb->gkey.clear();
    }
    CKS64(alloc64(pb, &pb->d_Ehist, (size_t)p.outer + 1));
    pb->Ehist_cap = p.outer + 1;
  }
  if (p.use_graph) {
    const std::vector<double> key = {double(p.outer), double(p.inner), double(lm), double(p.use_precond),
                                     p.lambda0, p.lambda_min, p.lambda_max, p.diag_min, p.diag_max,
                                     p.eta, p.rel_tol};
    if (!pb->gexec || key != pb->gkey) {
      if (pb->gexec) {
        cudaGraphExecDestroy(pb->gexec);
        pb->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK64(cudaStreamBeginCapture(pb->cap_stream, cudaStreamCaptureModeThreadLocal));
      const opt_status s = enqueue_solve64(pb, p, lm, pb->cap_stream);
      const cudaError_t e = cudaStreamEndCapture(pb->cap_stream, &g);
      if (s != OPT_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return fail64(e, "cudaStreamEndCapture");
      const cudaError_t e2 = cudaGraphInstantiate(&pb->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) return fail64(e2, "cudaGraphInstantiate");
      pb->gkey = key;
    }
    CK64(cudaEventRecord(pb->ev0, st));
    CK64(cudaGraphLaunch(pb->gexec, st));
    CK64(cudaEventRecord(pb->ev1, st));
  } else {
    CK64(cudaEventRecord(pb->ev0, st));
    CKS64(enqueue_solve64(pb, p, lm, st));
    CK64(cudaEventRecord(pb->ev1, st));
  }
  CK64(cudaEventSynchronize(pb->ev1));
  Scalars s;
  CK64(cudaMemcpy(&s, pb->d_s, sizeof(Scalars), cudaMemcpyDeviceToHost));
  const int outer_done = lm ? s.outer_done : p.outer;
  std::vector<double> eh;
  CKS64(download64(eh, pb->d_Ehist, (size_t)outer_done + 1));
  if (rep) {
    rep->outer_done = outer_done;
    rep->pcg_done = s.pcg_iters;
    rep->accepted = lm ? s.accepted_total : p.outer;
    rep->converged = s.converged;
    rep->E0 = eh[0];
    rep->E_final = eh[(size_t)outer_done];
    rep->lambda_final = lm ? s.lambda : 0.0;
    if (rep->E_history) std::memcpy(rep->E_history, eh.data(), eh.size() * sizeof(double));
    float ms = 0.f;
    CK64(cudaEventElapsedTime(&ms, pb->ev0, pb->ev1));
    rep->ms = ms;
  }
  if (s.nonfinite) return OPT_ERR_NUMERIC;
  return OPT_OK;
}

// PCGInit at the caller's x with damping lambda (hooks), on the default stream.
opt_status hook_init64(opt_problem_f64* pb, double lambda, double* jtf, double* diag, double* energy) {
  CK64(cudaDeviceSynchronize());
  P64 P = pb->hp;
  P.lm = lambda != 0.0 ? 1 : 0;
  P.use_precond = 1;
  P.Ehist = nullptr;
  P.jtf_out = jtf;
  P.diag_out = diag;
  CKS64(copy_x(pb, true, nullptr));
  k64_reset<<<1, 1>>>(pb->d_s, lambda);
  if (pb->kind != F64_POISSON) k64_rot<<<pb->nblk, NT>>>(P);
  k_init(pb, P, nullptr, -1, 1e-6, 1e32);
  CK64(cudaGetLastError());
  CK64(cudaDeviceSynchronize());
  if (energy) {
    Scalars s;
    CK64(cudaMemcpy(&s, pb->d_s, sizeof(s), cudaMemcpyDeviceToHost));
    *energy = s.E;
  }
  return OPT_OK;
}

opt_status finish_create64(std::unique_ptr<opt_problem_f64>& pb, opt_problem_f64** out) {
  CK64(cudaDeviceSynchronize());
  *out = pb.release();
  return OPT_OK;
}

}  // namespace

extern "C" {

opt_status opt_problem_create_grid_f64(const opt_grid_desc_f64* d, const opt_solve_params* params,
                                       opt_problem_f64** out) {
  (void)params;
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d || (d->kind != OPT_ARAP_WARP_2D && d->kind != OPT_POISSON_2D)) return OPT_ERR_INVALID_ARG;
  if (d->W < 1 || d->H < 1 || d->W >= 32768 || d->H >= 32768) return OPT_ERR_INVALID_ARG;
  const bool warp = d->kind == OPT_ARAP_WARP_2D;
  const int nx = warp ? 3 : 4, nc = warp ? 2 : 4;
  for (int c = 0; c < nx; ++c)
    if (!d->unknowns[c]) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < nc; ++c)
    if (!d->consts[c]) return OPT_ERR_INVALID_ARG;
  if (warp && (!(d->w_reg >= 0.0) || !(d->w_fit >= 0.0) || !std::isfinite(d->w_reg) || !std::isfinite(d->w_fit)))
    return OPT_ERR_INVALID_ARG;
  const long long n = (long long)d->W * d->H;
  std::unique_ptr<opt_problem_f64> pb(new opt_problem_f64());
  pb->kind = warp ? F64_WARP : F64_POISSON;
  pb->nx = nx;
  P64& P = pb->hp;
  P.kind = pb->kind;
  P.W = d->W;
  P.H = d->H;
  P.nx = nx;
  P.n = n;
  for (int c = 0; c < nx; ++c) pb->user_x[c] = d->unknowns[c];
  std::vector<double> consts((size_t)n * nc), tmp;
  for (int c = 0; c < nc; ++c) {
    CKS64(download64(tmp, d->consts[c], (size_t)n));
    std::copy(tmp.begin(), tmp.end(), consts.begin() + (size_t)c * n);
  }
  if (!all_finite(consts)) return OPT_ERR_INVALID_ARG;
  std::vector<int> hslot, hidx;
  std::vector<double> htgt;
  if (warp) {
    CKS64(handle_slots(d->handle_idx, d->n_handles, n, hslot, hidx));
    if (d->n_handles > 0) {
      if (!d->handle_target) return OPT_ERR_INVALID_ARG;
      CKS64(download64(htgt, d->handle_target, 2 * (size_t)d->n_handles));
      if (!all_finite(htgt)) return OPT_ERR_INVALID_ARG;
    }
  } else {
    hslot.assign((size_t)n, -1);
  }
  CKS64(plan_common(pb.get(), consts, hslot, htgt, warp ? d->w_reg : 1.0, warp ? d->w_fit : 0.0));
  if (warp) CKS64(alloc64(pb.get(), &P.G, 8 * (size_t)n));   // R'(theta) v per direction
  if (d->mask) {
    uint8_t* mk = nullptr;
    CKS64(alloc64(pb.get(), &mk, (size_t)n));
    CK64(cudaMemcpy(mk, d->mask, (size_t)n, cudaMemcpyDeviceToDevice));
    P.mask = mk;
  }
  return finish_create64(pb, out);
}

opt_status opt_problem_create_graph_f64(const opt_graph_desc_f64* d, const opt_solve_params* params,
                                        opt_problem_f64** out) {
  (void)params;
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d || d->V < 1 || d->E < 0 || (d->E > 0 && (!d->v0 || !d->v1))) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < 6; ++c)
    if (!d->unknowns[c]) return OPT_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c)
    if (!d->urshape[c]) return OPT_ERR_INVALID_ARG;
  if (!(d->w_reg >= 0.0) || !(d->w_fit >= 0.0) || !std::isfinite(d->w_reg) || !std::isfinite(d->w_fit))
    return OPT_ERR_INVALID_ARG;
  const int V = d->V, E = d->E;
  std::vector<int> e0, e1;
  CKS64(download64(e0, d->v0, (size_t)E));
  CKS64(download64(e1, d->v1, (size_t)E));
  for (int e = 0; e < E; ++e)
    if (e0[e] < 0 || e0[e] >= V || e1[e] < 0 || e1[e] >= V || e0[e] == e1[e]) return OPT_ERR_INVALID_ARG;
  // out-edges sorted by (v0, v1): counting sort by v1, then stable by v0
  std::vector<int> orow(V + 1, 0), irow(V + 1, 0), tmpo((size_t)E), oe1((size_t)E), isrc((size_t)E);
  std::vector<int> ieid((size_t)E);
  {
    std::vector<int> cnt(V + 1, 0);
    for (int e = 0; e < E; ++e) cnt[e1[e] + 1]++;
    for (int v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
    for (int e = 0; e < E; ++e) tmpo[cnt[e1[e]]++] = e;            // edges by v1
    for (int e = 0; e < E; ++e) orow[e0[e] + 1]++;
    for (int v = 0; v < V; ++v) orow[v + 1] += orow[v];
    std::vector<int> pos(orow.begin(), orow.end() - 1);
    for (int k = 0; k < E; ++k) {                                    // stable by v0
      const int e = tmpo[k];
      oe1[pos[e0[e]]++] = e1[e];
    }
    // in-edges of b from the (v0, v1)-sorted list: sources ascending
    for (int e = 0; e < E; ++e) irow[e1[e] + 1]++;
    for (int v = 0; v < V; ++v) irow[v + 1] += irow[v];
    std::vector<int> ipos(irow.begin(), irow.end() - 1);
    for (int a = 0; a < V; ++a)
      for (int k = orow[a]; k < orow[a + 1]; ++k) {
        const int slot = ipos[oe1[k]]++;
        isrc[slot] = a;
        ieid[slot] = k;
      }
  }
  std::unique_ptr<opt_problem_f64> pb(new opt_problem_f64());
  pb->kind = F64_MESH;
  pb->nx = 6;
  P64& P = pb->hp;
  P.kind = F64_MESH;
  P.W = 0;
  P.H = 0;
  P.nx = 6;
  P.n = V;
  P.ne = E;
  for (int c = 0; c < 6; ++c) pb->user_x[c] = d->unknowns[c];
  std::vector<double> consts((size_t)V * 3), tmp;
  for (int c = 0; c < 3; ++c) {
    CKS64(download64(tmp, d->urshape[c], (size_t)V));
    std::copy(tmp.begin(), tmp.end(), consts.begin() + (size_t)c * V);
  }
  if (!all_finite(consts)) return OPT_ERR_INVALID_ARG;
  std::vector<int> hslot, hidx;
  std::vector<double> htgt;
  CKS64(handle_slots(d->handle_idx, d->n_handles, V, hslot, hidx));
  if (d->n_handles > 0) {
    if (!d->handle_target) return OPT_ERR_INVALID_ARG;
    CKS64(download64(htgt, d->handle_target, 3 * (size_t)d->n_handles));
    if (!all_finite(htgt)) return OPT_ERR_INVALID_ARG;
  }
  CKS64(plan_common(pb.get(), consts, hslot, htgt, d->w_reg, d->w_fit));
  int *a = nullptr, *b = nullptr, *c2 = nullptr, *d2 = nullptr, *e2 = nullptr;
  CKS64(upload64(pb.get(), &a, orow));
  CKS64(upload64(pb.get(), &b, oe1));
  CKS64(upload64(pb.get(), &c2, irow));
  CKS64(upload64(pb.get(), &d2, isrc));
  CKS64(upload64(pb.get(), &e2, ieid));
  CKS64(alloc64(pb.get(), &P.G, 9 * (size_t)E));            // dR/dA_m w per directed edge
  P.orow = a;
  P.oe1 = b;
  P.irow = c2;
  P.isrc = d2;
  P.ieid = e2;
  return finish_create64(pb, out);
}

opt_status opt_problem_destroy_f64(opt_problem_f64* pb) {
  if (!pb) return OPT_OK;
  cudaDeviceSynchronize();
  delete pb;
  return OPT_OK;
}

opt_status opt_solve_gn_f64(opt_problem_f64* pb, const opt_solve_params* params, opt_report* report) {
  return run_solve64(pb, params, report, false);
}

opt_status opt_solve_lm_f64(opt_problem_f64* pb, const opt_solve_params* params, opt_report* report) {
  return run_solve64(pb, params, report, true);
}

opt_status opt_eval_jtf_f64(opt_problem_f64* pb, double* jtf, double* diag, double* energy) {
  if (!pb) return OPT_ERR_INVALID_ARG;
  return hook_init64(pb, 0.0, jtf, diag, energy);
}

opt_status opt_eval_energy_f64(opt_problem_f64* pb, double* energy) {
  if (!pb || !energy) return OPT_ERR_INVALID_ARG;
  CK64(cudaDeviceSynchronize());
  P64 P = pb->hp;
  P.Ehist = nullptr;
  CKS64(copy_x(pb, true, nullptr));
  k64_reset<<<1, 1>>>(pb->d_s, 0.0);
  k_energy(pb, P, nullptr, 0, -3);
  CK64(cudaGetLastError());
  Scalars s;
  CK64(cudaMemcpy(&s, pb->d_s, sizeof(s), cudaMemcpyDeviceToHost));
  *energy = s.E;
  return OPT_OK;
}

opt_status opt_apply_jtj_f64(opt_problem_f64* pb, const double* p, double* q, double lambda, double* pq) {
  if (!pb || !p || !q || !(lambda >= 0.0) || !std::isfinite(lambda)) return OPT_ERR_INVALID_ARG;
  CKS64(hook_init64(pb, lambda, nullptr, nullptr, nullptr));
  const size_t bytes = (size_t)pb->hp.n * pb->nx * sizeof(double);
  CK64(cudaMemcpy(pb->d_pin, p, bytes, cudaMemcpyDeviceToDevice));
  P64 P = pb->hp;
  P.lm = lambda != 0.0 ? 1 : 0;
  P.pin = pb->d_pin;
  P.Ehist = nullptr;
  k64_force_active<<<1, 1>>>(pb->d_s);
  k_apply(pb, P, nullptr, 0);
  CK64(cudaGetLastError());
  CK64(cudaMemcpy(q, P.q, bytes, cudaMemcpyDeviceToDevice));
  if (pq) {
    Scalars s;
    CK64(cudaMemcpy(&s, pb->d_s, sizeof(s), cudaMemcpyDeviceToHost));
    *pq = s.pq;
  }
  return OPT_OK;
}

opt_status opt_profile_pcg_f64(opt_problem_f64* pb, int32_t n_iters, void* stream, float* ms) {
  if (!pb || !ms || n_iters < 1 || n_iters > 100000) return OPT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK64(cudaStreamSynchronize(st));
  P64 P = pb->hp;
  P.lm = 0;
  P.use_precond = 1;
  P.Ehist = nullptr;
  CKS64(copy_x(pb, true, st));
  std::vector<cudaEvent_t> ev(2 + 4 * (size_t)n_iters);
  for (auto& e : ev) CK64(cudaEventCreate(&e));
  k64_reset<<<1, 1, 0, st>>>(pb->d_s, 0.0);
  CK64(cudaEventRecord(ev[0], st));
  k_rot(pb, st);
  k_init(pb, P, st, -1, 1e-6, 1e32);
  CK64(cudaEventRecord(ev[1], st));
  for (int i = 0; i < n_iters; ++i) {
    CK64(cudaEventRecord(ev[2 + 4 * i], st));
    k_apply(pb, P, st, i);
    CK64(cudaEventRecord(ev[3 + 4 * i], st));
    CK64(cudaEventRecord(ev[4 + 4 * i], st));
    k_update(pb, P, st);
    CK64(cudaEventRecord(ev[5 + 4 * i], st));
  }
  CK64(cudaGetLastError());
  CK64(cudaStreamSynchronize(st));
  float t = 0.f, ta = 0.f, tu = 0.f;
  CK64(cudaEventElapsedTime(&t, ev[0], ev[1]));
  for (int i = 0; i < n_iters; ++i) {
    float a = 0.f, u = 0.f;
    CK64(cudaEventElapsedTime(&a, ev[2 + 4 * i], ev[3 + 4 * i]));
    CK64(cudaEventElapsedTime(&u, ev[4 + 4 * i], ev[5 + 4 * i]));
    ta += a;
    tu += u;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  ms[0] = t;
  ms[1] = ta / n_iters;
  ms[2] = tu / n_iters;
  return OPT_OK;
}

opt_status opt_problem_info_f64(const opt_problem_f64* pb, int64_t* n_unknowns, int32_t* n_planes,
                                int64_t* plane_len) {
  if (!pb) return OPT_ERR_INVALID_ARG;
  if (n_unknowns) *n_unknowns = pb->hp.n * pb->nx;
  if (n_planes) *n_planes = pb->nx;
  if (plane_len) *plane_len = pb->hp.n;
  return OPT_OK;
}

opt_status opt_measure_fp64_fma_rate(void* stream, double* gflops) {
  if (!gflops) return OPT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CK64(cudaGetDevice(&dev));
  CK64(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, iters = 4096;
  double* out = nullptr;
  CK64(cudaMalloc(&out, (size_t)blocks * sizeof(double)));
  cudaEvent_t e0, e1;
  CK64(cudaEventCreate(&e0));
  CK64(cudaEventCreate(&e1));
  k64_fma_probe<<<blocks, NT, 0, st>>>(out, 64, 0.999999, 1e-7);   // warm-up
  CK64(cudaEventRecord(e0, st));
  k64_fma_probe<<<blocks, NT, 0, st>>>(out, iters, 0.999999, 1e-7);
  CK64(cudaEventRecord(e1, st));
  const cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return fail64(e, "opt_measure_fp64_fma_rate");
  const double flops = 2.0 * 8.0 * iters * (double)blocks * NT;
  *gflops = ms > 0.f ? flops / (ms * 1e-3) * 1e-9 : 0.0;
  return OPT_OK;
}


}  // extern "C"
