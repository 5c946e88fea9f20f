// Matrix-free graph kernels (Sec. 4.1 "Graph-based Array Access", Sec. 5.3.2).
//
// As in the paper, one thread owns one edge residual and scatters its
// contributions to the rows of the two vertices it touches (Fig. 11: a row of
// J p per residual, then J^T times it).  Edges are kept sorted by (v0, v1), so
// the v0-side contributions of a warp are first summed over each run of equal
// v0 (segmented shuffle reduction) and only the run head issues the atomic
// add; the v1 side issues one float32 atomic add per component.
//
// ARAP mesh algebra per edge e = (a, b), v = U_a - U_b, d = O - U:
//   r_e       = s_w [(d_a - d_b) + (v - R(A_a) v)]              (= Fig. 25)
//   dr/dd_a   = s_w I,  dr/dd_b = -s_w I,
//   dr/dA_a,m = g_m = -s_w (dR/dA_m)(A_a) v,  R = Rz(az) Ry(ay) Rx(ax).
//
// Per outer iteration (PCGInit): k_mesh_init_v (fit rows, zero accumulators),
// k_mesh_init_e (edge rows of J^T F, angle diagonal, energy), k_mesh_init_f
// (b, M^-1, r, delta, float64 r.z).  Per PCG iteration: k_mesh_apply_v
// (p = z + beta p, fit + damping rows of q), k_mesh_apply_e (edge rows of
// J^T J p, float64 p.q -> alpha), k_mesh_update (vector update -> beta).
#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

// Segment structure of a warp whose lanes hold sorted keys.
struct Seg {
  unsigned flags;   // bit k: lane + 2^k is in this lane's segment
  bool head;        // first lane of its segment within the warp
};

__device__ __forceinline__ Seg seg_info(int key) {
  const int lane = threadIdx.x & 31;
  Seg sg;
  sg.flags = 0u;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int off = 1 << k;
    const int other = __shfl_down_sync(0xffffffffu, key, off);
    if (lane + off < 32 && other == key) sg.flags |= 1u << k;
  }
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  sg.head = (lane == 0) || (prev != key);
  return sg;
}

// Sum of v over the lanes of this lane's segment at or after this lane
// (the full segment sum at the head lane).
__device__ __forceinline__ float seg_sum(float v, unsigned flags) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float o = __shfl_down_sync(0xffffffffu, v, 1 << k);
    if (flags & (1u << k)) v += o;
  }
  return v;
}

__device__ __forceinline__ int handle_of(const MeshProb& pr, int v) {
  const int t = v / VT;
  for (int h = pr.hbeg[t]; h < pr.hbeg[t + 1]; ++h)
    if (pr.hpix[h] == v) return h;
  return -1;
}

// ---------------------------------------------------------------------------
// PCGInit
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_mesh_init_v(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  const long long pl = pr.Vp;
  float e = 0.f;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    const int h = handle_of(pr, v);
    if (h >= 0) {
      const float f0 = pr.s_f * (pr.x[v] - pr.htgt[3 * h]);
      const float f1 = pr.s_f * (pr.x[pl + v] - pr.htgt[3 * h + 1]);
      const float f2 = pr.s_f * (pr.x[2 * pl + v] - pr.htgt[3 * h + 2]);
      g0 = pr.s_f * f0; g1 = pr.s_f * f1; g2 = pr.s_f * f2;
      e += f0 * f0 + f1 * f1 + f2 * f2;
    }
    pr.q[v] = g0; pr.q[pl + v] = g1; pr.q[2 * pl + v] = g2;
    pr.q[3 * pl + v] = 0.f; pr.q[4 * pl + v] = 0.f; pr.q[5 * pl + v] = 0.f;
    pr.acc[v] = 0.f; pr.acc[pl + v] = 0.f; pr.acc[2 * pl + v] = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      float sn, cs;
      sincosf(pr.x[(3 + m) * pl + v], &sn, &cs);
      pr.csn[(2 * m) * pl + v] = cs;
      pr.csn[(2 * m + 1) * pl + v] = sn;
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, e, 0.0, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) s->part0 = a;
  }
}

__global__ void __launch_bounds__(NT) k_mesh_init_e(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  float e = 0.f;
  for (int base = ch.begin; base < ch.end; base += NT) {
    const int ei = base + (int)threadIdx.x;
    const bool ok = ei < ch.end;
    const int a = ok ? pr.e0[ei] : -1;
    float c[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int b = 0;
    float rb0 = 0.f, rb1 = 0.f, rb2 = 0.f;
    if (ok) {
      b = pr.e1[ei];
      const float vx = pr.U[a] - pr.U[b];
      const float vy = pr.U[pl + a] - pr.U[pl + b];
      const float vz = pr.U[2 * pl + a] - pr.U[2 * pl + b];
      const RotV R = rot_apply_cs(pr.csn[a], pr.csn[pl + a], pr.csn[2 * pl + a], pr.csn[3 * pl + a],
                                    pr.csn[4 * pl + a], pr.csn[5 * pl + a], vx, vy, vz);
      const float r0 = sw * ((pr.x[a] - pr.x[b]) + (vx - R.rv[0]));
      const float r1 = sw * ((pr.x[pl + a] - pr.x[pl + b]) + (vy - R.rv[1]));
      const float r2 = sw * ((pr.x[2 * pl + a] - pr.x[2 * pl + b]) + (vz - R.rv[2]));
      c[0] = sw * r0; c[1] = sw * r1; c[2] = sw * r2;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float g0 = -sw * R.g[m][0], g1 = -sw * R.g[m][1], g2 = -sw * R.g[m][2];
        c[3 + m] = g0 * r0 + g1 * r1 + g2 * r2;
        c[6 + m] = g0 * g0 + g1 * g1 + g2 * g2;
      }
      rb0 = -sw * r0; rb1 = -sw * r1; rb2 = -sw * r2;
      e += r0 * r0 + r1 * r1 + r2 * r2;
    }
    const Seg sg = seg_info(a);
#pragma unroll
    for (int k = 0; k < 9; ++k) c[k] = seg_sum(c[k], sg.flags);
    if (ok && sg.head) {
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(&pr.q[k * pl + a], c[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k) atomicAdd(&pr.acc[k * pl + a], c[6 + k]);
    }
    if (ok) {
      atomicAdd(&pr.q[b], rb0);
      atomicAdd(&pr.q[pl + b], rb1);
      atomicAdd(&pr.q[2 * pl + b], rb2);
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, e, 0.0, &s->counter, pr.echunk_end - pr.echunk_begin)) {
    double a, b;
    gather_partials(part, pr.echunk_begin, pr.echunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) s->part1 = a;
  }
}

__global__ void __launch_bounds__(NT) k_mesh_init_f(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part, int k_outer,
                                                    float dmin, float dmax) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  const long long pl = pr.Vp;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  float rz = 0.f;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float dg[4];
    dg[0] = pr.degw[v];
    dg[1] = pr.acc[v]; dg[2] = pr.acc[pl + v]; dg[3] = pr.acc[2 * pl + v];
    float mv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float dcv;
      mv[k] = minv_entry(dg[k], lam, dmin, dmax, pr.use_precond, &dcv);
      pr.m[k * pl + v] = mv[k];
      if (pr.lm) pr.dc[k * pl + v] = dcv;
      if (pr.diag_out) pr.diag_out[k * pl + v] = dg[k];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float g = pr.q[c * pl + v];
      const float b = -g;
      pr.r[c * pl + v] = b;
      pr.d[c * pl + v] = 0.f;
      if (pr.jtf_out) pr.jtf_out[c * pl + v] = g;
      rz += b * (mv[c < 3 ? 0 : c - 2] * b);
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, rz, 0.0, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) {
      const double E = s->part0 + s->part1;
      s->rz = a;
      s->E = E;
      if (pr.Ehist && k_outer >= 0) pr.Ehist[k_outer] = E;
      s->beta_f = 0.f;
      s->pcg_active = (a != 0.0) && isfinite(a);
      if (!isfinite(a) || !isfinite(E)) s->nonfinite = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// PCGStep: applyJTJ
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ld4g(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float c4(const float4& a, int k) {
  return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w));
}

// Direction update and the vertex rows of q (fit + damping), four vertices per
// thread: every load of a quad is issued before any store.  Vertex ranges
// start at multiples of 256 and the planes are padded to 32 (zeros), so a quad
// never leaves the plane.
__global__ void __launch_bounds__(NT) k_mesh_apply_v(const MeshProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     double* __restrict__ part,
                                                     const float* __restrict__ p_override, int par,
                                                     int update) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float beta = s->beta_f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const float* __restrict__ pin = p_override ? p_override : pr.p + (long long)(par & 1) * 6 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 6 * pl;
  float acc = 0.f;
  const int q0 = ch.begin / 4, q1 = (ch.end + 3) / 4;
  for (int qi = q0 + threadIdx.x; qi < q1; qi += NT) {
    const int v0 = 4 * qi;
    float4 pv[6];
    if (update) {
      float4 rr[6], mm[4], po[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) rr[c] = ld4g(pr.r + c * pl + v0);
#pragma unroll
      for (int k = 0; k < 4; ++k) mm[k] = ld4g(pr.m + k * pl + v0);
      if (beta != 0.0f) {
#pragma unroll
        for (int c = 0; c < 6; ++c) po[c] = ld4g(pin + c * pl + v0);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float4 m = mm[c < 3 ? 0 : c - 2];
        pv[c] = make_float4(m.x * rr[c].x, m.y * rr[c].y, m.z * rr[c].z, m.w * rr[c].w);
        if (beta != 0.0f) {
          pv[c].x = fmaf(beta, po[c].x, pv[c].x); pv[c].y = fmaf(beta, po[c].y, pv[c].y);
          pv[c].z = fmaf(beta, po[c].z, pv[c].z); pv[c].w = fmaf(beta, po[c].w, pv[c].w);
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) *reinterpret_cast<float4*>(pout + c * pl + v0) = pv[c];
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) pv[c] = ld4g(pin + c * pl + v0);
    }
    float4 dc[4];
    if (pr.lm) {
#pragma unroll
      for (int k = 0; k < 4; ++k) dc[k] = ld4g(pr.dc + k * pl + v0);
    }
    float q[6][4];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) q[c][k] = pr.lm ? lam * c4(dc[c < 3 ? 0 : c - 2], k) * c4(pv[c], k) : 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int v = v0 + k;
      if (v < pr.V && handle_of(pr, v) >= 0) {
        q[0][k] += pr.w_fit * c4(pv[0], k);
        q[1][k] += pr.w_fit * c4(pv[1], k);
        q[2][k] += pr.w_fit * c4(pv[2], k);
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      *reinterpret_cast<float4*>(pr.q + c * pl + v0) = make_float4(q[c][0], q[c][1], q[c][2], q[c][3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc += c4(pv[c], k) * q[c][k];
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) s->part0 = a;
  }
}

// Edge rows of J^T J p; p.q = p^T (fit + damping) p + sum_e |J_e p|^2.
__global__ void __launch_bounds__(NT) k_mesh_apply_e(const MeshProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     double* __restrict__ part,
                                                     const float* __restrict__ p_override, int par) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  const float* __restrict__ p = p_override ? p_override : pr.p + (long long)((par + 1) & 1) * 6 * pl;
  float acc = 0.f;
  for (int base = ch.begin; base < ch.end; base += NT) {
    const int ei = base + (int)threadIdx.x;
    const bool ok = ei < ch.end;
    const int a = ok ? pr.e0[ei] : -1;
    float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int b = 0;
    float jb0 = 0.f, jb1 = 0.f, jb2 = 0.f;
    if (ok) {
      b = pr.e1[ei];
      const float vx = pr.U[a] - pr.U[b];
      const float vy = pr.U[pl + a] - pr.U[pl + b];
      const float vz = pr.U[2 * pl + a] - pr.U[2 * pl + b];
      const RotV R = rot_apply_cs(pr.csn[a], pr.csn[pl + a], pr.csn[2 * pl + a], pr.csn[3 * pl + a],
                                    pr.csn[4 * pl + a], pr.csn[5 * pl + a], vx, vy, vz);
      const float pa3 = p[3 * pl + a], pa4 = p[4 * pl + a], pa5 = p[5 * pl + a];
      float j0 = sw * (p[a] - p[b]);
      float j1 = sw * (p[pl + a] - p[pl + b]);
      float j2 = sw * (p[2 * pl + a] - p[2 * pl + b]);
      float g[3][3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        g[m][0] = -sw * R.g[m][0]; g[m][1] = -sw * R.g[m][1]; g[m][2] = -sw * R.g[m][2];
      }
      j0 += g[0][0] * pa3 + g[1][0] * pa4 + g[2][0] * pa5;
      j1 += g[0][1] * pa3 + g[1][1] * pa4 + g[2][1] * pa5;
      j2 += g[0][2] * pa3 + g[1][2] * pa4 + g[2][2] * pa5;
      c[0] = sw * j0; c[1] = sw * j1; c[2] = sw * j2;
#pragma unroll
      for (int m = 0; m < 3; ++m) c[3 + m] = g[m][0] * j0 + g[m][1] * j1 + g[m][2] * j2;
      jb0 = -sw * j0; jb1 = -sw * j1; jb2 = -sw * j2;
      acc += j0 * j0 + j1 * j1 + j2 * j2;
    }
    const Seg sg = seg_info(a);
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = seg_sum(c[k], sg.flags);
    if (ok && sg.head) {
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(&pr.q[k * pl + a], c[k]);
    }
    if (ok) {
      atomicAdd(&pr.q[b], jb0);
      atomicAdd(&pr.q[pl + b], jb1);
      atomicAdd(&pr.q[2 * pl + b], jb2);
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.echunk_end - pr.echunk_begin)) {
    double a, b;
    gather_partials(part, pr.echunk_begin, pr.echunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) {
      const double pq = s->part0 + a;
      s->pq = pq;
      if (pq > 0.0 && isfinite(pq)) {
        s->alpha_f = (float)(s->rz / pq);
      } else {
        s->alpha_f = 0.f;
        s->pcg_active = 0;
        if (!isfinite(pq)) s->nonfinite = 1;
      }
    }
  }
}

// delta += alpha p, r -= alpha q, z = M^-1 r, float64 r.z -> beta; four
// vertices per thread, all loads first.
__global__ void __launch_bounds__(NT) k_mesh_update(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part, int par) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float alpha = s->alpha_f;
  const float* __restrict__ pn = pr.p + (long long)((par + 1) & 1) * 6 * pl;
  float acc = 0.f;
  const int q0 = ch.begin / 4, q1 = (ch.end + 3) / 4;
  for (int qi = q0 + threadIdx.x; qi < q1; qi += NT) {
    const int v0 = 4 * qi;
    float4 pv[6], qv[6], dv[6], rv[6], mv[4];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      pv[c] = ld4g(pn + c * pl + v0);
      qv[c] = ld4g(pr.q + c * pl + v0);
      dv[c] = *reinterpret_cast<const float4*>(pr.d + c * pl + v0);
      rv[c] = *reinterpret_cast<const float4*>(pr.r + c * pl + v0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) mv[k] = ld4g(pr.m + k * pl + v0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float4 m = mv[c < 3 ? 0 : c - 2];
      dv[c].x += alpha * pv[c].x; dv[c].y += alpha * pv[c].y;
      dv[c].z += alpha * pv[c].z; dv[c].w += alpha * pv[c].w;
      rv[c].x -= alpha * qv[c].x; rv[c].y -= alpha * qv[c].y;
      rv[c].z -= alpha * qv[c].z; rv[c].w -= alpha * qv[c].w;
      acc += rv[c].x * (m.x * rv[c].x) + rv[c].y * (m.y * rv[c].y) + rv[c].z * (m.z * rv[c].z) +
             rv[c].w * (m.w * rv[c].w);
      *reinterpret_cast<float4*>(pr.d + c * pl + v0) = dv[c];
      *reinterpret_cast<float4*>(pr.r + c * pl + v0) = rv[c];
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double rz, unused;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, rz, unused);
    if (threadIdx.x == 0) {
      s->beta_f = (float)(rz / s->rz);
      s->rz = rz;
      s->pcg_iters += 1;
      if (rz == 0.0 || !isfinite(rz)) s->pcg_active = 0;
      if (!isfinite(rz)) s->nonfinite = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// energies and the outer update
// ---------------------------------------------------------------------------
// Fit part: mode 0 -> part0 = E_fit(x); mode 1 -> part0 = E_fit(x + delta)
// (the fit residual is linear, so the model value is the same).
__global__ void __launch_bounds__(NT) k_mesh_energy_v(const MeshProb* __restrict__ probs,
                                                      const Chunk* __restrict__ chunks,
                                                      double* __restrict__ part, int mode) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  const long long pl = pr.Vp;
  float e = 0.f;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    const int h = handle_of(pr, v);
    if (h < 0) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float dv = pr.x[c * pl + v];
      if (mode == 1) dv += pr.d[c * pl + v];
      const float f = pr.s_f * (dv - pr.htgt[3 * h + c]);
      e += f * f;
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, e, 0.0, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) s->part0 = a;
  }
}

__global__ void __launch_bounds__(NT) k_mesh_energy_e(const MeshProb* __restrict__ probs,
                                                      const Chunk* __restrict__ chunks,
                                                      double* __restrict__ part, int mode,
                                                      int hist_idx) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  float e0 = 0.f, e1 = 0.f;
  for (int ei = ch.begin + threadIdx.x; ei < ch.end; ei += NT) {
    const int a = pr.e0[ei], b = pr.e1[ei];
    const float vx = pr.U[a] - pr.U[b];
    const float vy = pr.U[pl + a] - pr.U[pl + b];
    const float vz = pr.U[2 * pl + a] - pr.U[2 * pl + b];
    const float dd0 = pr.x[a] - pr.x[b], dd1 = pr.x[pl + a] - pr.x[pl + b];
    const float dd2 = pr.x[2 * pl + a] - pr.x[2 * pl + b];
    const RotV R = rot_apply(pr.x[3 * pl + a], pr.x[4 * pl + a], pr.x[5 * pl + a], vx, vy, vz);
    const float r0 = sw * (dd0 + (vx - R.rv[0]));
    const float r1 = sw * (dd1 + (vy - R.rv[1]));
    const float r2 = sw * (dd2 + (vz - R.rv[2]));
    if (mode == 0) {
      e0 += r0 * r0 + r1 * r1 + r2 * r2;
    } else {
      const float ea0 = pr.d[a] - pr.d[b], ea1 = pr.d[pl + a] - pr.d[pl + b];
      const float ea2 = pr.d[2 * pl + a] - pr.d[2 * pl + b];
      const float t3 = pr.d[3 * pl + a], t4 = pr.d[4 * pl + a], t5 = pr.d[5 * pl + a];
      const RotV R2 = rot_apply(pr.x[3 * pl + a] + t3, pr.x[4 * pl + a] + t4, pr.x[5 * pl + a] + t5, vx, vy, vz);
      const float u0 = sw * ((dd0 + ea0) + (vx - R2.rv[0]));
      const float u1 = sw * ((dd1 + ea1) + (vy - R2.rv[1]));
      const float u2 = sw * ((dd2 + ea2) + (vz - R2.rv[2]));
      e0 += u0 * u0 + u1 * u1 + u2 * u2;
      const float l0 = r0 + sw * ea0 - sw * (R.g[0][0] * t3 + R.g[1][0] * t4 + R.g[2][0] * t5);
      const float l1 = r1 + sw * ea1 - sw * (R.g[0][1] * t3 + R.g[1][1] * t4 + R.g[2][1] * t5);
      const float l2 = r2 + sw * ea2 - sw * (R.g[0][2] * t3 + R.g[1][2] * t4 + R.g[2][2] * t5);
      e1 += l0 * l0 + l1 * l1 + l2 * l2;
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, e0, e1, &s->counter, pr.echunk_end - pr.echunk_begin)) {
    double a, b;
    gather_partials(part, pr.echunk_begin, pr.echunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) {
      if (mode == 0) {
        const double E = s->part0 + a;
        s->E = E;
        const int k = hist_idx >= 0 ? hist_idx : (hist_idx == -1 ? s->outer_done : -1);
        if (pr.Ehist && k >= 0) pr.Ehist[k] = E;
        if (!isfinite(E)) s->nonfinite = 1;
      } else {
        s->E_trial = s->part0 + a;
        s->model = s->part0 + b;
      }
    }
  }
}

__global__ void __launch_bounds__(NT) k_mesh_step(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks, int cond) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  if (cond && !pr.s->accept) return;
  if (!cond && pr.s->done) return;
  const long long pl = pr.Vp;
  float* __restrict__ x = pr.x;
  const float* __restrict__ d = pr.d;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float xv[6], dv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { xv[c] = x[c * pl + v]; dv[c] = __ldg(d + c * pl + v); }
#pragma unroll
    for (int c = 0; c < 6; ++c) x[c * pl + v] = xv[c] + dv[c];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_mesh_init(const MeshLaunch& L, int k_outer, float dmin, float dmax) {
  launch_pdl(k_mesh_init_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part);
  launch_pdl(k_mesh_init_e, L.nechunks, NT, 0, L.stream, L.probs, L.echunks, L.part);
  launch_pdl(k_mesh_init_f, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, k_outer, dmin, dmax);
}

void launch_mesh_apply(const MeshLaunch& L, const float* p_override, int par, int update) {
  launch_pdl(k_mesh_apply_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, p_override, par, update);
  launch_pdl(k_mesh_apply_e, L.nechunks, NT, 0, L.stream, L.probs, L.echunks, L.part, p_override, par);
}

void launch_mesh_update(const MeshLaunch& L, int par) {
  launch_pdl(k_mesh_update, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, par);
}

void launch_mesh_energy(const MeshLaunch& L, int mode, int hist_idx) {
  launch_pdl(k_mesh_energy_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, mode);
  launch_pdl(k_mesh_energy_e, L.nechunks, NT, 0, L.stream, L.probs, L.echunks, L.part, mode, hist_idx);
}

void launch_mesh_step(const MeshLaunch& L, int cond) {
  launch_pdl(k_mesh_step, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, cond);
}

}  // namespace optgb
