// Embedded deformation (Fig. 28, Appendix A.2.1): every vertex carries a
// displacement d (position O = U + d) and a full 3x3 matrix R (row-major,
// 12 unknowns per vertex); soft constraints keep R a rotation.  Residuals:
//   edge e = (a, b), w = U_a - U_b:   s_w [(d_a - d_b) + w - R_a w]
//     dr/dd_a = s_w I, dr/dd_b = -s_w I, dr_i/dR_a[3i + c] = -s_w w_c;
//   vertex, columns c_k = (R[k], R[3+k], R[6+k]):
//     s_r c0.c1, s_r c0.c2, s_r c1.c2, s_r (c0.c0 - 1), s_r (c1.c1 - 1), s_r (c2.c2 - 1)
//     d(c_i.c_j)/dc_i = c_j, d(c_i.c_i)/dc_i = 2 c_i;
//   handle h: s_f (O_h - C_h).
// (Fig. 28 writes the edge residual as (O_b - O_a) - R_a (U_b - U_a), the
// negation of the one above: the same energy and the same J^T J, J^T F.)
//
// Same gather design as the ARAP mesh kernels: a thread owns a vertex and
// walks its out-edges (own edge rows: displacement and matrix) and its
// in-edges (far-end displacement rows), plus its six constraint rows, so
// every row of J^T F / J^T J p is summed by one thread in a fixed order, no
// atomics.  Neighbour data comes from per-vertex records: grec[v] = (U, 0)
// and three float4 of the 12-vector, vrec[3v .. 3v+2] = x (PCGInit, energy)
// or p (applyJTJ), in unknown order (d0 d1 d2 R00 | R01 R02 R10 R11 | R12 R20
// R21 R22).  The Jacobi diagonal keeps 10 planes: one shared by the three
// displacement rows (w_reg * degree + w_fit, planned) and one per matrix
// entry.
#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

constexpr int NXE = 12;   // unknowns per vertex
constexpr int NME = 10;   // distinct-diagonal planes
constexpr int KBE = 6;    // neighbour indices fetched ahead per vertex (icosphere degree 5 / 6)

// Visits the out-edge targets e1[o0 .. o1) (or in-edge sources) of a vertex:
// the first KBE indices are loaded together before any neighbour record is
// needed, the rest of a longer row one by one.
template <typename F>
__device__ __forceinline__ void for_neighbours(const int* __restrict__ idx, int o0, int o1, F&& f) {
  int j[KBE];
#pragma unroll
  for (int t = 0; t < KBE; ++t) j[t] = o0 + t < o1 ? __ldg(idx + o0 + t) : 0;
#pragma unroll
  for (int t = 0; t < KBE; ++t)
    if (o0 + t < o1) f(j[t]);
  for (int k = o0 + KBE; k < o1; ++k) f(__ldg(idx + k));
}

__device__ __forceinline__ int mplane_e(int c) { return c < 3 ? 0 : c - 2; }

__device__ __forceinline__ int handle_of_e(const MeshProb& pr, int v) {
  const int t = v / VT;
  for (int h = pr.hbeg[t]; h < pr.hbeg[t + 1]; ++h)
    if (pr.hpix[h] == v) return h;
  return -1;
}

__device__ __forceinline__ void load12(const float4* rec, int v, float (&o)[NXE]) {
  const float4 a = rec[3 * v], b = rec[3 * v + 1], c = rec[3 * v + 2];
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  o[8] = c.x; o[9] = c.y; o[10] = c.z; o[11] = c.w;
}
__device__ __forceinline__ void store12(float4* rec, int v, const float (&o)[NXE]) {
  rec[3 * v] = make_float4(o[0], o[1], o[2], o[3]);
  rec[3 * v + 1] = make_float4(o[4], o[5], o[6], o[7]);
  rec[3 * v + 2] = make_float4(o[8], o[9], o[10], o[11]);
}

// The six constraint values (c0.c1, c0.c2, c1.c2, c0.c0 - 1, c1.c1 - 1,
// c2.c2 - 1) of the matrix m[9] (row-major), unscaled.
__device__ __forceinline__ void col_constraints(const float* m, float (&f)[6]) {
  float d01 = 0.f, d02 = 0.f, d12 = 0.f, d00 = 0.f, d11 = 0.f, d22 = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float c0 = m[3 * r], c1 = m[3 * r + 1], c2 = m[3 * r + 2];
    d01 += c0 * c1; d02 += c0 * c2; d12 += c1 * c2;
    d00 += c0 * c0; d11 += c1 * c1; d22 += c2 * c2;
  }
  f[0] = d01; f[1] = d02; f[2] = d12; f[3] = d00 - 1.f; f[4] = d11 - 1.f; f[5] = d22 - 1.f;
}

// Linearised constraints J_rot t of a matrix direction t[9] at m[9], unscaled.
__device__ __forceinline__ void col_constraints_lin(const float* m, const float* t, float (&f)[6]) {
  float a01 = 0.f, a02 = 0.f, a12 = 0.f, a00 = 0.f, a11 = 0.f, a22 = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float c0 = m[3 * r], c1 = m[3 * r + 1], c2 = m[3 * r + 2];
    const float t0 = t[3 * r], t1 = t[3 * r + 1], t2 = t[3 * r + 2];
    a01 += c1 * t0 + c0 * t1; a02 += c2 * t0 + c0 * t2; a12 += c2 * t1 + c1 * t2;
    a00 += c0 * t0; a11 += c1 * t1; a22 += c2 * t2;
  }
  f[0] = a01; f[1] = a02; f[2] = a12; f[3] = 2.f * a00; f[4] = 2.f * a11; f[5] = 2.f * a22;
}

// out[9] += J_rot^T y for the six constraint values y (unscaled).
__device__ __forceinline__ void col_constraints_t(const float* m, const float (&y)[6], float* out) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float c0 = m[3 * r], c1 = m[3 * r + 1], c2 = m[3 * r + 2];
    out[3 * r] += c1 * y[0] + c2 * y[1] + 2.f * c0 * y[3];
    out[3 * r + 1] += c0 * y[0] + c2 * y[2] + 2.f * c1 * y[4];
    out[3 * r + 2] += c0 * y[1] + c1 * y[2] + 2.f * c2 * y[5];
  }
}

// ---------------------------------------------------------------------------
// PCGInit
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_ed_init_v(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  if (pr.s->done) return;
  const long long pl = pr.Vp;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float x[NXE];
#pragma unroll
    for (int c = 0; c < NXE; ++c) x[c] = pr.x[c * pl + v];
    store12(pr.vrec, v, x);
    pr.grec[v] = make_float4(__ldg(pr.U + v), __ldg(pr.U + pl + v), __ldg(pr.U + 2 * pl + v), 0.f);
  }
}

// Gather pass: J^T F, diag(J^T J), the energy of the vertex's own rows
// (out-edges, constraints, fit), then b = -J^T F, M^-1, r = b, delta = 0.
// resident blocks per SM the gather PCGInit is compiled for (64 registers, a
// few spills that stay in L1; measured against 2 and 3 at level 9: 362 / 393 -> 355 us)
#ifndef ED_INIT_MIN_BLOCKS
#define ED_INIT_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(NT, ED_INIT_MIN_BLOCKS) k_ed_init_pull(const MeshProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     double* __restrict__ part, int k_outer, float dmin,
                                                     float dmax) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w, sr = pr.s_r, w = pr.w_reg;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  F2 acc_rz = f2_zero(), acc_E = f2_zero();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += NT) {
    float xi[NXE];
    load12(pr.vrec, i, xi);
    const float4 ui = __ldg(pr.grec + i);
    float g[NXE], dR[9];
#pragma unroll
    for (int c = 0; c < NXE; ++c) g[c] = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) dR[k] = 0.f;
    float e = 0.f;
    const int h = handle_of_e(pr, i);
    if (h >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float f = pr.s_f * (xi[c] - pr.htgt[3 * h + c]);
        g[c] += pr.s_f * f;
        e += f * f;
      }
    }
    for_neighbours(pr.e1, pr.orow[i], pr.orow[i + 1], [&](int j) {
      const float4 dj = pr.vrec[3 * j];
      const float4 uj = __ldg(pr.grec + j);
      const float wv[3] = {ui.x - uj.x, ui.y - uj.y, ui.z - uj.z};
      const float dd[3] = {xi[0] - dj.x, xi[1] - dj.y, xi[2] - dj.z};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float rw = xi[3 + 3 * r] * wv[0] + xi[4 + 3 * r] * wv[1] + xi[5 + 3 * r] * wv[2];
        const float f = sw * ((dd[r] + wv[r]) - rw);
        e += f * f;
        g[r] += sw * f;
#pragma unroll
        for (int c = 0; c < 3; ++c) g[3 + 3 * r + c] -= sw * wv[c] * f;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float wc2 = w * wv[c] * wv[c];
        dR[c] += wc2; dR[3 + c] += wc2; dR[6 + c] += wc2;
      }
    });
    for_neighbours(pr.isrc, pr.irow[i], pr.irow[i + 1], [&](int j) {
      float xj[NXE];
      load12(pr.vrec, j, xj);
      const float4 uj = __ldg(pr.grec + j);
      const float wv[3] = {uj.x - ui.x, uj.y - ui.y, uj.z - ui.z};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float rw = xj[3 + 3 * r] * wv[0] + xj[4 + 3 * r] * wv[1] + xj[5 + 3 * r] * wv[2];
        g[r] -= sw * (sw * (((xj[r] - xi[r]) + wv[r]) - rw));
      }
    });
    {
      float f[6];
      col_constraints(xi + 3, f);
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        f[t] *= sr;
        e += f[t] * f[t];
        f[t] *= sr;                 // J^T carries another s_r
      }
      col_constraints_t(xi + 3, f, g + 3);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float c0 = xi[3 + 3 * r], c1 = xi[4 + 3 * r], c2 = xi[5 + 3 * r];
        const float wr = pr.w_rot;
        dR[3 * r] += wr * (c1 * c1 + c2 * c2 + 4.f * c0 * c0);
        dR[3 * r + 1] += wr * (c0 * c0 + c2 * c2 + 4.f * c1 * c1);
        dR[3 * r + 2] += wr * (c0 * c0 + c1 * c1 + 4.f * c2 * c2);
      }
    }
    float mv[NME];
#pragma unroll
    for (int k = 0; k < NME; ++k) {
      const float dg = k == 0 ? pr.degw[i] : dR[k - 1];
      float dcv;
      mv[k] = minv_entry(dg, lam, dmin, dmax, pr.use_precond, &dcv);
      pr.m[k * pl + i] = mv[k];
      if (pr.lm) pr.dc[k * pl + i] = dcv;
      if (pr.diag_out) pr.diag_out[k * pl + i] = dg;
    }
#pragma unroll
    for (int c = 0; c < NXE; ++c) {
      const float b = -g[c];
      pr.r[c * pl + i] = b;
      pr.d[c * pl + i] = 0.f;
      if (pr.jtf_out) pr.jtf_out[c * pl + i] = g[c];
      f2_add_prod(acc_rz, b, __fmul_rn(mv[mplane_e(c)], b));
    }
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
// Direction update p = z + beta p (or p = p_override), written to the planes
// and the records.
__global__ void __launch_bounds__(NT) k_ed_apply_v(const MeshProb* __restrict__ probs,
                                                   const Chunk* __restrict__ chunks,
                                                   const float* __restrict__ p_override, int par, int update) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float beta = s->beta_f;
  const float* __restrict__ pin = p_override ? p_override : pr.p + (long long)(par & 1) * NXE * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * NXE * pl;
  const float* __restrict__ rr = pr.r;
  const float* __restrict__ mm = pr.m;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float pv[NXE];
    if (update) {
      // every load before any store (the planes may not alias, but the
      // compiler cannot know: stores first would serialise the loads)
      float rv[NXE], mv[NME], po[NXE];
#pragma unroll
      for (int c = 0; c < NXE; ++c) {
        rv[c] = __ldcg(rr + c * pl + v);
        po[c] = beta != 0.0f ? __ldcg(pin + c * pl + v) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < NME; ++k) mv[k] = __ldg(mm + k * pl + v);
#pragma unroll
      for (int c = 0; c < NXE; ++c) pv[c] = fmaf(beta, po[c], mv[mplane_e(c)] * rv[c]);
#pragma unroll
      for (int c = 0; c < NXE; ++c) pout[c * pl + v] = pv[c];
    } else {
#pragma unroll
      for (int c = 0; c < NXE; ++c) pv[c] = pin[c * pl + v];
    }
    store12(pr.vrec, v, pv);
  }
}

// Gather pass: q_i = (fit + damping) p_i + own edge rows + incoming edge
// rows + constraint rows, float64 p.q -> alpha.
__global__ void __launch_bounds__(NT) k_ed_apply_pull(const MeshProb* __restrict__ probs,
                                                      const Chunk* __restrict__ chunks,
                                                      double* __restrict__ part) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float wreg = pr.w_reg;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  F2 acc = f2_zero();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += NT) {
    float pi[NXE], q[NXE];
    load12(pr.vrec, i, pi);
    const float4 ui = __ldg(pr.grec + i);
#pragma unroll
    for (int c = 0; c < NXE; ++c) q[c] = pr.lm ? lam * pr.dc[mplane_e(c) * pl + i] * pi[c] : 0.f;
    if (handle_of_e(pr, i) >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] += pr.w_fit * pi[c];
    }
    // (plain loops: prefetching the indices as PCGInit does costs this
    // kernel occupancy -- 100 instead of 80 registers -- and was measured slower)
    for (int k = pr.orow[i]; k < pr.orow[i + 1]; ++k) {
      const int j = pr.e1[k];
      const float4 pj = pr.vrec[3 * j];
      const float4 uj = __ldg(pr.grec + j);
      const float wv[3] = {ui.x - uj.x, ui.y - uj.y, ui.z - uj.z};
      const float pd[3] = {pi[0] - pj.x, pi[1] - pj.y, pi[2] - pj.z};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        // J p / s_w of row r; J^T (J p) carries s_w^2 = w_reg
        const float jp = pd[r] - (pi[3 + 3 * r] * wv[0] + pi[4 + 3 * r] * wv[1] + pi[5 + 3 * r] * wv[2]);
        q[r] += wreg * jp;
#pragma unroll
        for (int c = 0; c < 3; ++c) q[3 + 3 * r + c] -= wreg * wv[c] * jp;
      }
    }
    for (int k = pr.irow[i]; k < pr.irow[i + 1]; ++k) {
      const int j = pr.isrc[k];
      float pj[NXE];
      load12(pr.vrec, j, pj);
      const float4 uj = __ldg(pr.grec + j);
      const float wv[3] = {uj.x - ui.x, uj.y - ui.y, uj.z - ui.z};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float jp = (pj[r] - pi[r]) - (pj[3 + 3 * r] * wv[0] + pj[4 + 3 * r] * wv[1] + pj[5 + 3 * r] * wv[2]);
        q[r] -= wreg * jp;
      }
    }
    {
      float m9[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) m9[k] = pr.x[(3 + k) * pl + i];
      float y[6];
      col_constraints_lin(m9, pi + 3, y);
#pragma unroll
      for (int t = 0; t < 6; ++t) y[t] *= pr.w_rot;
      col_constraints_t(m9, y, q + 3);
    }
#pragma unroll
    for (int c = 0; c < NXE; ++c) {
      pr.q[c * pl + i] = q[c];
      f2_add_prod(acc, pi[c], q[c]);
    }
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

// delta += alpha p, r -= alpha q, z = M^-1 r, float64 r.z -> beta.
// The update streams twelve planes per array: in two groups of six unknowns
// (all loads of a group before its stores) it fits 64 registers and runs 4
// blocks per SM; loading all twelve first took 186 registers (one block per
// SM).  Measured at icosphere level 9: 173 -> 143 us (level-7 LM solve 27.5 ->
// 24.1 ms); the summation order of r.z is unchanged.
#ifndef ED_UPDATE_MIN_BLOCKS
#define ED_UPDATE_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(NT, ED_UPDATE_MIN_BLOCKS) k_ed_update(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  double* __restrict__ part, int par) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float alpha = s->alpha_f;
  const float* __restrict__ pn = pr.p + (long long)((par + 1) & 1) * NXE * pl;
  float* __restrict__ dd = pr.d;
  float* __restrict__ rr = pr.r;
  const float* __restrict__ qq = pr.q;
  const float* __restrict__ mm = pr.m;
  F2 acc = f2_zero();
#ifndef ED_UPDATE_GROUPS
#define ED_UPDATE_GROUPS 2
#endif
  constexpr int GC = NXE / ED_UPDATE_GROUPS;   // unknowns per group
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
#pragma unroll 1
    for (int g0 = 0; g0 < NXE; g0 += GC) {
      // every load of the group before any of its stores
      float pv[GC], qv[GC], dv[GC], rv[GC], mv[GC];
#pragma unroll
      for (int k = 0; k < GC; ++k) {
        const int c = g0 + k;
        pv[k] = __ldcg(pn + c * pl + v);
        qv[k] = __ldcg(qq + c * pl + v);
        dv[k] = dd[c * pl + v];
        rv[k] = rr[c * pl + v];
        mv[k] = __ldg(mm + mplane_e(c) * pl + v);
      }
#pragma unroll
      for (int k = 0; k < GC; ++k) {
        dv[k] = fmaf(alpha, pv[k], dv[k]);
        rv[k] = fmaf(-alpha, qv[k], rv[k]);
        f2_add_prod(acc, rv[k], __fmul_rn(mv[k], rv[k]));
      }
#pragma unroll
      for (int k = 0; k < GC; ++k) {
        dd[(g0 + k) * pl + v] = dv[k];
        rr[(g0 + k) * pl + v] = rv[k];
      }
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
// E(x) (mode 0) or E(x + delta) and |F(x) + J(x) delta|^2 (mode 1); every
// residual is evaluated by the vertex that owns it (its out-edges, its
// constraints, its fit term).
__global__ void __launch_bounds__(NT) k_ed_energy(const MeshProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  double* __restrict__ part, int mode, int hist_idx) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  const long long pl = pr.Vp;
  const float sw = pr.s_w, sr = pr.s_r;
  F2 acc0 = f2_zero(), acc1 = f2_zero();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += NT) {
    float e0 = 0.f, e1 = 0.f;           // this vertex's residuals
    float xi[NXE], di[NXE];
#pragma unroll
    for (int c = 0; c < NXE; ++c) {
      xi[c] = pr.x[c * pl + i];
      di[c] = mode == 1 ? pr.d[c * pl + i] : 0.f;
    }
    const float ui[3] = {pr.U[i], pr.U[pl + i], pr.U[2 * pl + i]};
    const int h = handle_of_e(pr, i);
    if (h >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float f = pr.s_f * (xi[c] + di[c] - pr.htgt[3 * h + c]);   // linear: trial == model
        e0 += f * f;
        e1 += f * f;
      }
    }
    for (int k = pr.orow[i]; k < pr.orow[i + 1]; ++k) {
      const int j = pr.e1[k];
      const float wv[3] = {ui[0] - pr.U[j], ui[1] - pr.U[pl + j], ui[2] - pr.U[2 * pl + j]};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float dd = xi[r] - pr.x[r * pl + j];
        const float rw = xi[3 + 3 * r] * wv[0] + xi[4 + 3 * r] * wv[1] + xi[5 + 3 * r] * wv[2];
        const float f = sw * ((dd + wv[r]) - rw);
        if (mode == 0) {
          e0 += f * f;
        } else {
          const float ed = di[r] - pr.d[r * pl + j];
          const float tw = di[3 + 3 * r] * wv[0] + di[4 + 3 * r] * wv[1] + di[5 + 3 * r] * wv[2];
          const float t = sw * (((dd + ed) + wv[r]) - (rw + tw));
          const float l = f + sw * (ed - tw);
          e0 += t * t;
          e1 += l * l;
        }
      }
    }
    float f[6];
    col_constraints(xi + 3, f);
    if (mode == 0) {
#pragma unroll
      for (int t = 0; t < 6; ++t) e0 += (sr * f[t]) * (sr * f[t]);
    } else {
      float xt[9], lin[6], ft[6];
#pragma unroll
      for (int k = 0; k < 9; ++k) xt[k] = xi[3 + k] + di[3 + k];
      col_constraints(xt, ft);
      col_constraints_lin(xi + 3, di + 3, lin);
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        e0 += (sr * ft[t]) * (sr * ft[t]);
        const float l = sr * (f[t] + lin[t]);
        e1 += l * l;
      }
    }
    f2_add(acc0, e0);
    f2_add(acc1, e1);
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc0, acc1, &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
    double a, b;
    gather_partials(part, pr.vchunk_begin, pr.vchunk_end, &s->counter, a, b);
    if (threadIdx.x == 0) {
      if (mode == 0) {
        s->E = a;
        const int k = hist_idx >= 0 ? hist_idx : (hist_idx == -1 ? s->outer_done : -1);
        if (pr.Ehist && k >= 0) pr.Ehist[k] = a;
        if (!isfinite(a)) s->nonfinite = 1;
      } else {
        s->E_trial = a;
        s->model = b;
      }
    }
  }
}

__global__ void __launch_bounds__(NT) k_ed_step(const MeshProb* __restrict__ probs,
                                                const Chunk* __restrict__ chunks, int cond) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  if (cond && !pr.s->accept) return;
  if (!cond && pr.s->done) return;
  const long long pl = pr.Vp;
  float* __restrict__ x = pr.x;
  const float* __restrict__ dd = pr.d;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float xv[NXE], dv[NXE];
#pragma unroll
    for (int c = 0; c < NXE; ++c) {
      xv[c] = x[c * pl + v];
      dv[c] = __ldg(dd + c * pl + v);
    }
#pragma unroll
    for (int c = 0; c < NXE; ++c) x[c * pl + v] = xv[c] + dv[c];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (called by the launch_mesh_* dispatchers for dim == 12)
// ---------------------------------------------------------------------------
void launch_ed_init(const MeshLaunch& L, int k_outer, float dmin, float dmax) {
  launch_pdl(k_ed_init_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks);
  launch_pdl(k_ed_init_pull, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, k_outer, dmin, dmax);
}
void launch_ed_apply(const MeshLaunch& L, const float* p_override, int par, int update) {
  launch_pdl(k_ed_apply_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, p_override, par, update);
  launch_pdl(k_ed_apply_pull, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part);
}
void launch_ed_update(const MeshLaunch& L, int par) {
  launch_pdl(k_ed_update, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, par);
}
void launch_ed_energy(const MeshLaunch& L, int mode, int hist_idx) {
  launch_pdl(k_ed_energy, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, mode, hist_idx);
}
void launch_ed_step(const MeshLaunch& L, int cond) {
  launch_pdl(k_ed_step, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, cond);
}

}  // namespace optgb
