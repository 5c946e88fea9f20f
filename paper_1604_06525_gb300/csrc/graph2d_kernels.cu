// ARAP image warping on an explicit graph (Sec. 4.1 "Graph-based Array
// Access"; the explicit-graph side of the implicit-grid vs explicit-graph
// comparison, Fig. 18).  Per vertex: displacement (dx, dy) and angle theta,
// rest position U; per directed edge e = (a, b), v = U_a - U_b:
//   r_e       = s_w [(d_a - d_b) + (v - R(theta_a) v)]          (= Fig. 24)
//   dr/dd_a   = s_w I,  dr/dd_b = -s_w I,
//   dr/dtheta_a = g = -s_w R'(theta_a) v = s_w G_a,
//   G = (s v_x + c v_y, s v_y - c v_x),  R counter-clockwise.
// Fit rows s_f (O_h - C_h) per handle.
//
// Same gather design as the mesh kernels: a thread owns a vertex and walks
// its out-edges (own rows: displacement and angle) and its in-edges (far-end
// displacement rows); neighbour data comes from one 16-byte record per
// vertex for the geometry, grec[v] = (U_x, U_y, cos theta, sin theta), and
// one for the 3-vector, vrec[v] = (x or p: dx, dy, theta, 0).
#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

__device__ __forceinline__ int handle_of2(const MeshProb& pr, int v) {
  const int t = v / VT;
  for (int h = pr.hbeg[t]; h < pr.hbeg[t + 1]; ++h)
    if (pr.hpix[h] == v) return h;
  return -1;
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float cc4(const float4& a, int k) {
  return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w));
}

// ---------------------------------------------------------------------------
// PCGInit
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_wg_init_v(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  if (pr.s->done) return;
  const long long pl = pr.Vp;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    const float dx = pr.x[v], dy = pr.x[pl + v], th = pr.x[2 * pl + v];
    float sn, cs;
    sincosf(th, &sn, &cs);
    pr.grec[v] = make_float4(__ldg(pr.U + v), __ldg(pr.U + pl + v), cs, sn);
    pr.vrec[v] = make_float4(dx, dy, th, 0.f);
  }
}

// Gather pass: J^T F (fit, own residuals with their angle row, incoming
// residuals), diag(J^T J) (displacement: planned w_reg * degree + w_fit;
// angle: sum |g|^2 over the out-edges), the energy of the own residuals;
// b = -J^T F, M^-1, r = b, delta = 0, float64 r.z and E.
__global__ void __launch_bounds__(NT) k_wg_init_pull(const MeshProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     double* __restrict__ part, int k_outer, float dmin,
                                                     float dmax) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  F2 acc_rz = f2_zero(), acc_E = f2_zero();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += NT) {
    const float4 xi = pr.vrec[i];
    const float4 gi = __ldg(pr.grec + i);
    float g0 = 0.f, g1 = 0.f, gt = 0.f, dt = 0.f, e = 0.f;
    const int h = handle_of2(pr, i);
    if (h >= 0) {
      const float f0 = pr.s_f * (xi.x - pr.htgt[2 * h]), f1 = pr.s_f * (xi.y - pr.htgt[2 * h + 1]);
      g0 += pr.s_f * f0;
      g1 += pr.s_f * f1;
      e += f0 * f0 + f1 * f1;
    }
    for (int k = pr.orow[i]; k < pr.orow[i + 1]; ++k) {
      const int j = pr.e1[k];
      const float4 xj = pr.vrec[j];
      const float4 gj = __ldg(pr.grec + j);
      const float vx = gi.x - gj.x, vy = gi.y - gj.y;
      const float Gx = fmaf(gi.w, vx, gi.z * vy), Gy = fmaf(gi.w, vy, -gi.z * vx);
      // v - R v = (v_x + G_y, v_y - G_x)
      const float r0 = sw * ((xi.x - xj.x) + (vx + Gy));
      const float r1 = sw * ((xi.y - xj.y) + (vy - Gx));
      g0 += sw * r0;
      g1 += sw * r1;
      gt += sw * (Gx * r0 + Gy * r1);
      dt += sw * sw * (Gx * Gx + Gy * Gy);
      e += r0 * r0 + r1 * r1;
    }
    for (int k = pr.irow[i]; k < pr.irow[i + 1]; ++k) {
      const int j = pr.isrc[k];
      const float4 xj = pr.vrec[j];
      const float4 gj = __ldg(pr.grec + j);
      const float vx = gj.x - gi.x, vy = gj.y - gi.y;
      const float Gx = fmaf(gj.w, vx, gj.z * vy), Gy = fmaf(gj.w, vy, -gj.z * vx);
      g0 -= sw * (sw * ((xj.x - xi.x) + (vx + Gy)));
      g1 -= sw * (sw * ((xj.y - xi.y) + (vy - Gx)));
    }
    float dcd, dct;
    const float dd = pr.degw[i];
    const float md = minv_entry(dd, lam, dmin, dmax, pr.use_precond, &dcd);
    const float mt = minv_entry(dt, lam, dmin, dmax, pr.use_precond, &dct);
    pr.m[i] = md;
    pr.m[pl + i] = mt;
    if (pr.lm) { pr.dc[i] = dcd; pr.dc[pl + i] = dct; }
    if (pr.diag_out) { pr.diag_out[i] = dd; pr.diag_out[pl + i] = dt; }
    pr.r[i] = -g0; pr.r[pl + i] = -g1; pr.r[2 * pl + i] = -gt;
    pr.d[i] = 0.f; pr.d[pl + i] = 0.f; pr.d[2 * pl + i] = 0.f;
    if (pr.jtf_out) { pr.jtf_out[i] = g0; pr.jtf_out[pl + i] = g1; pr.jtf_out[2 * pl + i] = gt; }
    f2_add_prod(acc_rz, g0, __fmul_rn(md, g0));
    f2_add_prod(acc_rz, g1, __fmul_rn(md, g1));
    f2_add_prod(acc_rz, gt, __fmul_rn(mt, gt));
    f2_add(acc_E, e);
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc_rz, acc_E, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double rz, E;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, rz, E);
    if (threadIdx.x == 0) {
      s->rz = rz;
      s->E = E;
      if (pr.Ehist && k_outer >= 0) pr.Ehist[k_outer] = E;
      s->beta_f = 0.f;
      s->pcg_active = (rz != 0.0) && isfinite(rz);
      if (!isfinite(rz) || !isfinite(E)) s->nonfinite = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// PCGStep: applyJTJ
// ---------------------------------------------------------------------------
// Direction update p = z + beta p (or p = p_override), four vertices per
// thread from the planes, written to the planes and to the records.
__global__ void __launch_bounds__(NT) k_wg_apply_v(const MeshProb* __restrict__ probs,
                                                   const Chunk* __restrict__ chunks,
                                                   const float* __restrict__ p_override, int par, int update) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float beta = s->beta_f;
  const float* __restrict__ pin = p_override ? p_override : pr.p + (long long)(par & 1) * 3 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 3 * pl;
  const int q0 = ch.begin / 4, q1 = (ch.end + 3) / 4;
  for (int qi = q0 + threadIdx.x; qi < q1; qi += NT) {
    const int v0 = 4 * qi;
    float4 pv[3];
    if (update) {
      float4 rr[3], po[3];
      const float4 md = ldg4(pr.m + v0), mt = ldg4(pr.m + pl + v0);
#pragma unroll
      for (int c = 0; c < 3; ++c) rr[c] = ldg4(pr.r + c * pl + v0);
      if (beta != 0.0f) {
#pragma unroll
        for (int c = 0; c < 3; ++c) po[c] = ldg4(pin + c * pl + v0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 m = c < 2 ? md : mt;
        pv[c] = make_float4(m.x * rr[c].x, m.y * rr[c].y, m.z * rr[c].z, m.w * rr[c].w);
        if (beta != 0.0f) {
          pv[c].x = fmaf(beta, po[c].x, pv[c].x); pv[c].y = fmaf(beta, po[c].y, pv[c].y);
          pv[c].z = fmaf(beta, po[c].z, pv[c].z); pv[c].w = fmaf(beta, po[c].w, pv[c].w);
        }
        *reinterpret_cast<float4*>(pout + c * pl + v0) = pv[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) pv[c] = ldg4(pin + c * pl + v0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int v = v0 + k;
      if (v < pr.V) pr.vrec[v] = make_float4(cc4(pv[0], k), cc4(pv[1], k), cc4(pv[2], k), 0.f);
    }
  }
}

// Gather pass: q_i = (fit + damping) p_i + sum over out-edges (i, j) of the own
// rows s_w J_e p (displacement) and g . J_e p (angle) + sum over in-edges
// (j, i) of -s_w J_e p (displacement), J_e p = s_w (p_a,d - p_b,d) + g p_a,t;
// float64 p.q -> alpha.
__global__ void __launch_bounds__(NT) k_wg_apply_pull(const MeshProb* __restrict__ probs,
                                                      const Chunk* __restrict__ chunks,
                                                      double* __restrict__ part) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  F2 acc = f2_zero();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += NT) {
    const float4 pi = pr.vrec[i];
    const float4 gi = __ldg(pr.grec + i);
    float q0 = 0.f, q1 = 0.f, qt = 0.f;
    if (pr.lm) {
      const float dd = lam * pr.dc[i], dt = lam * pr.dc[pl + i];
      q0 = dd * pi.x; q1 = dd * pi.y; qt = dt * pi.z;
    }
    if (handle_of2(pr, i) >= 0) { q0 += pr.w_fit * pi.x; q1 += pr.w_fit * pi.y; }
    for (int k = pr.orow[i]; k < pr.orow[i + 1]; ++k) {
      const int j = pr.e1[k];
      const float4 pj = pr.vrec[j];
      const float4 gj = __ldg(pr.grec + j);
      const float vx = gi.x - gj.x, vy = gi.y - gj.y;
      const float Gx = fmaf(gi.w, vx, gi.z * vy), Gy = fmaf(gi.w, vy, -gi.z * vx);
      // J_e p / s_w = (p_a,d - p_b,d) + G p_a,t
      const float j0 = fmaf(Gx, pi.z, pi.x - pj.x), j1 = fmaf(Gy, pi.z, pi.y - pj.y);
      q0 += sw * sw * j0;
      q1 += sw * sw * j1;
      qt += sw * sw * (Gx * j0 + Gy * j1);
    }
    for (int k = pr.irow[i]; k < pr.irow[i + 1]; ++k) {
      const int j = pr.isrc[k];
      const float4 pj = pr.vrec[j];
      const float4 gj = __ldg(pr.grec + j);
      const float vx = gj.x - gi.x, vy = gj.y - gi.y;
      const float Gx = fmaf(gj.w, vx, gj.z * vy), Gy = fmaf(gj.w, vy, -gj.z * vx);
      q0 -= sw * sw * fmaf(Gx, pj.z, pj.x - pi.x);
      q1 -= sw * sw * fmaf(Gy, pj.z, pj.y - pi.y);
    }
    pr.q[i] = q0; pr.q[pl + i] = q1; pr.q[2 * pl + i] = qt;
    f2_add_prod(acc, pi.x, q0);
    f2_add_prod(acc, pi.y, q1);
    f2_add_prod(acc, pi.z, qt);
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double pq, unused;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, pq, unused);
    if (threadIdx.x == 0) {
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
__global__ void __launch_bounds__(NT) k_wg_update(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  double* __restrict__ part, int par) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float alpha = s->alpha_f;
  const float* __restrict__ pn = pr.p + (long long)((par + 1) & 1) * 3 * pl;
  F2 acc = f2_zero();
  const int q0 = ch.begin / 4, q1 = (ch.end + 3) / 4;
  for (int qi = q0 + threadIdx.x; qi < q1; qi += NT) {
    const int v0 = 4 * qi;
    float4 pv[3], qv[3], dv[3], rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pv[c] = __ldcg(reinterpret_cast<const float4*>(pn + c * pl + v0));
      qv[c] = __ldcg(reinterpret_cast<const float4*>(pr.q + c * pl + v0));
      dv[c] = *reinterpret_cast<const float4*>(pr.d + c * pl + v0);
      rv[c] = *reinterpret_cast<const float4*>(pr.r + c * pl + v0);
    }
    const float4 md = ldg4(pr.m + v0), mt = ldg4(pr.m + pl + v0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 m = c < 2 ? md : mt;
      dv[c].x += alpha * pv[c].x; dv[c].y += alpha * pv[c].y;
      dv[c].z += alpha * pv[c].z; dv[c].w += alpha * pv[c].w;
      rv[c].x -= alpha * qv[c].x; rv[c].y -= alpha * qv[c].y;
      rv[c].z -= alpha * qv[c].z; rv[c].w -= alpha * qv[c].w;
      f2_add_prod(acc, rv[c].x, __fmul_rn(m.x, rv[c].x));
      f2_add_prod(acc, rv[c].y, __fmul_rn(m.y, rv[c].y));
      f2_add_prod(acc, rv[c].z, __fmul_rn(m.z, rv[c].z));
      f2_add_prod(acc, rv[c].w, __fmul_rn(m.w, rv[c].w));
      *reinterpret_cast<float4*>(pr.d + c * pl + v0) = dv[c];
      *reinterpret_cast<float4*>(pr.r + c * pl + v0) = rv[c];
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
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
// (= the fit part of |F + J delta|^2, the fit residual being linear).
__global__ void __launch_bounds__(NT) k_wg_energy_v(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part, int mode) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  const long long pl = pr.Vp;
  F2 e = f2_zero();
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    const int h = handle_of2(pr, v);
    if (h < 0) continue;
    float ev = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float dv = pr.x[c * pl + v];
      if (mode == 1) dv += pr.d[c * pl + v];
      const float f = pr.s_f * (dv - pr.htgt[2 * h + c]);
      ev += f * f;
    }
    f2_add(e, ev);
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, e, f2_zero(), &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) s->part0 = a;
  }
}

// Edge part: mode 0 -> E(x); mode 1 -> E(x + delta) and |F + J delta|^2.
__global__ void __launch_bounds__(NT) k_wg_energy_e(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    double* __restrict__ part, int mode, int hist_idx) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  F2 e0 = f2_zero(), e1 = f2_zero();
  for (int ei = ch.begin + threadIdx.x; ei < ch.end; ei += NT) {
    const int a = pr.e0[ei], b = pr.e1[ei];
    const float vx = pr.U[a] - pr.U[b], vy = pr.U[pl + a] - pr.U[pl + b];
    const float dd0 = pr.x[a] - pr.x[b], dd1 = pr.x[pl + a] - pr.x[pl + b];
    const float th = pr.x[2 * pl + a];
    float sn, cs;
    sincosf(th, &sn, &cs);
    const float Gx = fmaf(sn, vx, cs * vy), Gy = fmaf(sn, vy, -cs * vx);
    const float r0 = sw * (dd0 + (vx + Gy)), r1 = sw * (dd1 + (vy - Gx));
    if (mode == 0) {
      f2_add(e0, r0 * r0 + r1 * r1);
    } else {
      const float ea0 = pr.d[a] - pr.d[b], ea1 = pr.d[pl + a] - pr.d[pl + b], t = pr.d[2 * pl + a];
      float sn2, cs2;
      sincosf(th + t, &sn2, &cs2);
      const float G2x = fmaf(sn2, vx, cs2 * vy), G2y = fmaf(sn2, vy, -cs2 * vx);
      const float u0 = sw * ((dd0 + ea0) + (vx + G2y)), u1 = sw * ((dd1 + ea1) + (vy - G2x));
      f2_add(e0, u0 * u0 + u1 * u1);
      const float l0 = r0 + sw * fmaf(Gx, t, ea0), l1 = r1 + sw * fmaf(Gy, t, ea1);
      f2_add(e1, l0 * l0 + l1 * l1);
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

__global__ void __launch_bounds__(NT) k_wg_step(const MeshProb* __restrict__ probs,
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
    float xv[3], dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) { xv[c] = x[c * pl + v]; dv[c] = __ldg(d + c * pl + v); }
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * pl + v] = xv[c] + dv[c];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (called by the launch_mesh_* dispatchers for dim == 2)
// ---------------------------------------------------------------------------
void launch_wg_init(const MeshLaunch& L, int k_outer, float dmin, float dmax) {
  launch_pdl(k_wg_init_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks);
  launch_pdl(k_wg_init_pull, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, k_outer, dmin, dmax);
}

void launch_wg_apply(const MeshLaunch& L, const float* p_override, int par, int update) {
  launch_pdl(k_wg_apply_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, p_override, par, update);
  launch_pdl(k_wg_apply_pull, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part);
}

void launch_wg_update(const MeshLaunch& L, int par) {
  launch_pdl(k_wg_update, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, par);
}

void launch_wg_energy(const MeshLaunch& L, int mode, int hist_idx) {
  launch_pdl(k_wg_energy_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, mode);
  launch_pdl(k_wg_energy_e, L.nechunks, NT, 0, L.stream, L.probs, L.echunks, L.part, mode, hist_idx);
}

void launch_wg_step(const MeshLaunch& L, int cond) {
  launch_pdl(k_wg_step, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, cond);
}

}  // namespace optgb
