// Matrix-free graph kernels (Sec. 4.1 "Graph-based Array Access", Sec. 5.3.2).
//
// The paper maps one thread to one edge residual and scatters its
// contributions to the rows of the two vertices with atomics (Fig. 11).  Here
// every row of J^T F, diag(J^T J) and J^T J p is gathered instead: one thread
// owns one vertex i and walks
//   * its out-edges (i, j) (edges sorted by (v0, v1) -> CSR rows): the
//     residual's own rows at i (displacement and angles), and
//   * its in-edges (j, i) (a transposed list built at planning): the
//     residual's rows at its far end, the displacement rows of i,
// so each edge residual is evaluated twice (once from each end) and no
// atomic or cross-thread sum is needed; every row is summed in a fixed
// order.  What a thread reads of a neighbour sits in two per-vertex records
// (array of structures, a few 32-byte sectors per gather instead of one
// sector per plane):
//   grec[v] = (U_x, U_y, U_z, cos a_x), (sin a_x, cos a_y, sin a_y, cos a_z),
//             (sin a_z, 0, 0, 0)          written by PCGInit's vertex pass
//   vrec[v] = the vertex's 6-vector (x in PCGInit, p in applyJTJ), 2 float4
//
// ARAP mesh algebra per edge e = (a, b), v = U_a - U_b, d = O - U:
//   r_e       = s_w [(d_a - d_b) + (v - R(A_a) v)]              (= Fig. 25)
//   dr/dd_a   = s_w I,  dr/dd_b = -s_w I,
//   dr/dA_a,m = g_m = -s_w (dR/dA_m)(A_a) v,  R = Rz(az) Ry(ay) Rx(ax).
//
// Per outer iteration (PCGInit): k_mesh_init_v (cos / sin of the angles, the
// records), k_mesh_init_pull (J^T F, diag, M^-1, r, delta, float64 r.z and E).
// Per PCG iteration: k_mesh_apply_v (p = z + beta p into the planes and the
// records), k_mesh_apply_pull (J^T J p + fit + damping, float64 p.q -> alpha),
// k_mesh_update (vector update -> beta).
#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

__device__ __forceinline__ int handle_of(const MeshProb& pr, int v) {
  const int t = v / VT;
  for (int h = pr.hbeg[t]; h < pr.hbeg[t + 1]; ++h)
    if (pr.hpix[h] == v) return h;
  return -1;
}

constexpr int KB = 6;             // neighbour indices fetched ahead per vertex (icosphere degree 5 / 6)
#ifndef MESH_PULL_MIN_BLOCKS
#define MESH_PULL_MIN_BLOCKS 4    // resident blocks per SM the gather apply is compiled for
#endif

__device__ __forceinline__ float4 ld4g(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float c4(const float4& a, int k) {
  return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w));
}

// The 7-point stencil of a W x H x D voxel grid (volumetric problems): the
// six neighbour offsets in ascending order -- the order the sorted edge lists
// give -- and which of them lie inside the grid.
struct Stencil3 {
  int off[6];
  bool ok[6];
};
__device__ __forceinline__ Stencil3 stencil3(const MeshProb& pr, int i) {
  const int W = pr.gw, H = pr.gh, WH = W * H;
  const int x = i % W, y = (i / W) % H, z = i / WH;
  Stencil3 st;
  st.off[0] = -WH; st.ok[0] = z > 0;
  st.off[1] = -W;  st.ok[1] = y > 0;
  st.off[2] = -1;  st.ok[2] = x > 0;
  st.off[3] = 1;   st.ok[3] = x + 1 < W;
  st.off[4] = W;   st.ok[4] = y + 1 < H;
  st.off[5] = WH;  st.ok[5] = z + 1 < pr.gd;
  return st;
}

// A vertex's geometry record and 6-vector record.
struct GeoRec {
  float U[3];
  float cs[6];      // cos ax, sin ax, cos ay, sin ay, cos az, sin az
};
__device__ __forceinline__ GeoRec load_geo(const float4* __restrict__ grec, int v) {
  const float4 a = __ldg(grec + 3 * v), b = __ldg(grec + 3 * v + 1), c = __ldg(grec + 3 * v + 2);
  GeoRec g;
  g.U[0] = a.x; g.U[1] = a.y; g.U[2] = a.z;
  g.cs[0] = a.w; g.cs[1] = b.x; g.cs[2] = b.y; g.cs[3] = b.z; g.cs[4] = b.w; g.cs[5] = c.x;
  return g;
}
// 6-vector record written in the same launch chain (plain loads, not the
// read-only path)
__device__ __forceinline__ void load_vec(const float4* vrec, int v, float (&o)[6]) {
  const float4 a = vrec[2 * v], b = vrec[2 * v + 1];
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
}
__device__ __forceinline__ void load_vec3(const float4* vrec, int v, float (&o)[3]) {
  const float4 a = vrec[2 * v];
  o[0] = a.x; o[1] = a.y; o[2] = a.z;
}

// ---------------------------------------------------------------------------
// PCGInit
// ---------------------------------------------------------------------------
// Vertex pass: cos / sin of the angles and both records of every vertex.
__global__ void __launch_bounds__(NT) k_mesh_init_v(const MeshProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  if (pr.s->done) return;
  const long long pl = pr.Vp;
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    float x[6], U[3], cs[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) x[c] = pr.x[c * pl + v];
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c] = __ldg(pr.U + c * pl + v);
#pragma unroll
    for (int m = 0; m < 3; ++m) sincosf(x[3 + m], &cs[2 * m + 1], &cs[2 * m]);
    pr.grec[3 * v] = make_float4(U[0], U[1], U[2], cs[0]);
    pr.grec[3 * v + 1] = make_float4(cs[1], cs[2], cs[3], cs[4]);
    pr.grec[3 * v + 2] = make_float4(cs[5], 0.f, 0.f, 0.f);
    pr.vrec[2 * v] = make_float4(x[0], x[1], x[2], x[3]);
    pr.vrec[2 * v + 1] = make_float4(x[4], x[5], 0.f, 0.f);
  }
}

// Gather pass: per vertex i the rows of J^T F (fit, own edge residuals with
// their angle rows, incoming edge residuals), diag(J^T J) (displacement:
// planned w_reg * degree + w_fit; angles: sum |g_m|^2 over the out-edges),
// the energy of the own residuals, then b = -J^T F, M^-1, r = b, delta = 0.
// resident blocks per SM the gather PCGInit is compiled for (85 registers;
// measured against 2 and 4: level-9 PCGInit 330 -> 316 us, level 7 39.8 -> 36.1 us)
#ifndef MESH_INIT_MIN_BLOCKS
#define MESH_INIT_MIN_BLOCKS 3
#endif
template <bool G3>
__global__ void __launch_bounds__(NT, MESH_INIT_MIN_BLOCKS) k_mesh_init_pull(const MeshProb* __restrict__ probs,
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
    float xi[6];
    load_vec(pr.vrec, i, xi);
    const GeoRec gi = load_geo(pr.grec, i);
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // J^T F
    float da[3] = {0.f, 0.f, 0.f};                 // angle diagonal
    float e = 0.f;
    const int h = handle_of(pr, i);
    if (h >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float f = pr.s_f * (xi[c] - pr.htgt[3 * h + c]);
        g[c] += pr.s_f * f;
        e += f * f;
      }
    }
    auto own_edge = [&](int j) {
      float xj[3];
      load_vec3(pr.vrec, j, xj);
      const float4 uj = __ldg(pr.grec + 3 * j);
      const float vx = gi.U[0] - uj.x, vy = gi.U[1] - uj.y, vz = gi.U[2] - uj.z;
      const RotV R = rot_apply_cs(gi.cs[0], gi.cs[1], gi.cs[2], gi.cs[3], gi.cs[4], gi.cs[5], vx, vy, vz);
      const float r0 = sw * ((xi[0] - xj[0]) + (vx - R.rv[0]));
      const float r1 = sw * ((xi[1] - xj[1]) + (vy - R.rv[1]));
      const float r2 = sw * ((xi[2] - xj[2]) + (vz - R.rv[2]));
      g[0] += sw * r0; g[1] += sw * r1; g[2] += sw * r2;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float g0 = -sw * R.g[m][0], g1 = -sw * R.g[m][1], g2 = -sw * R.g[m][2];
        g[3 + m] += g0 * r0 + g1 * r1 + g2 * r2;
        da[m] += g0 * g0 + g1 * g1 + g2 * g2;
      }
      e += r0 * r0 + r1 * r1 + r2 * r2;
    };
    auto in_edge = [&](int j) {
      float xj[3];
      load_vec3(pr.vrec, j, xj);
      const GeoRec gj = load_geo(pr.grec, j);
      const float vx = gj.U[0] - gi.U[0], vy = gj.U[1] - gi.U[1], vz = gj.U[2] - gi.U[2];
      const RotV R = rot_apply_cs(gj.cs[0], gj.cs[1], gj.cs[2], gj.cs[3], gj.cs[4], gj.cs[5], vx, vy, vz);
      g[0] -= sw * (sw * ((xj[0] - xi[0]) + (vx - R.rv[0])));
      g[1] -= sw * (sw * ((xj[1] - xi[1]) + (vy - R.rv[1])));
      g[2] -= sw * (sw * ((xj[2] - xi[2]) + (vz - R.rv[2])));
    };
    if (G3) {
      const Stencil3 st = stencil3(pr, i);
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (st.ok[t]) own_edge(i + st.off[t]);
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (st.ok[t]) in_edge(i + st.off[t]);
    } else {
      for (int k = pr.orow[i]; k < pr.orow[i + 1]; ++k) own_edge(pr.e1[k]);
      for (int k = pr.irow[i]; k < pr.irow[i + 1]; ++k) in_edge(pr.isrc[k]);
    }
    const float dg[4] = {pr.degw[i], da[0], da[1], da[2]};
    float mv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float dcv;
      mv[k] = minv_entry(dg[k], lam, dmin, dmax, pr.use_precond, &dcv);
      pr.m[k * pl + i] = mv[k];
      if (pr.lm) pr.dc[k * pl + i] = dcv;
      if (pr.diag_out) pr.diag_out[k * pl + i] = dg[k];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float b = -g[c];
      pr.r[c * pl + i] = b;
      pr.d[c * pl + i] = 0.f;
      if (pr.jtf_out) pr.jtf_out[c * pl + i] = g[c];
      f2_add_prod(acc_rz, b, __fmul_rn(mv[c < 3 ? 0 : c - 2], b));
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
// Direction update p = z + beta p (or p = p_override), four vertices per
// thread from the planes (every load of a quad before any store), written to
// the planes and to the 6-vector records.  Vertex ranges start at multiples
// of 256 and the planes are padded to 32 (zeros), so a quad never leaves the
// plane; records are written for real vertices only.
__global__ void __launch_bounds__(NT) k_mesh_apply_v(const MeshProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     const float* __restrict__ p_override, int par,
                                                     int update) {
  pdl_begin();
  const Chunk ch = chunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl = pr.Vp;
  const float beta = s->beta_f;
  const float* __restrict__ pin = p_override ? p_override : pr.p + (long long)(par & 1) * 6 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 6 * pl;
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
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int v = v0 + k;
      if (v < pr.V) {
        pr.vrec[2 * v] = make_float4(c4(pv[0], k), c4(pv[1], k), c4(pv[2], k), c4(pv[3], k));
        pr.vrec[2 * v + 1] = make_float4(c4(pv[4], k), c4(pv[5], k), 0.f, 0.f);
      }
    }
  }
}

// Gather pass: q_i = (fit + damping) p_i + sum over out-edges (i, j) of the
// own rows s_w J_e p (displacement) and g_m . J_e p (angles) + sum over
// in-edges (j, i) of -s_w J_e p (displacement), with
//   J_e p = s_w (p_a,d - p_b,d) + sum_m g_m p_a,m   for e = (a, b);
// float64 p.q -> alpha.  The neighbour indices of the first KB out- and
// in-edges are loaded together before any record is needed; the kernel is
// bound by these dependent load chains, so it is compiled for
// MESH_PULL_MIN_BLOCKS resident blocks per SM (measured best at 4).
template <bool G3>
__global__ void __launch_bounds__(NT, MESH_PULL_MIN_BLOCKS) k_mesh_apply_pull(const MeshProb* __restrict__ probs,
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
    int o0 = 0, o1 = 0, n0 = 0, n1 = 0;
    int jo[KB], ji[KB];
    if (!G3) {
      o0 = pr.orow[i]; o1 = pr.orow[i + 1];
      n0 = pr.irow[i]; n1 = pr.irow[i + 1];
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        jo[t] = o0 + t < o1 ? pr.e1[o0 + t] : 0;
        ji[t] = n0 + t < n1 ? pr.isrc[n0 + t] : 0;
      }
    }
    float pi[6];
    load_vec(pr.vrec, i, pi);
    const GeoRec gi = load_geo(pr.grec, i);
    float q[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) q[c] = pr.lm ? lam * pr.dc[(c < 3 ? 0 : c - 2) * pl + i] * pi[c] : 0.f;
    if (handle_of(pr, i) >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] += pr.w_fit * pi[c];
    }
    auto own_edge = [&](int j) {
      float pj[3];
      load_vec3(pr.vrec, j, pj);
      const float4 uj = __ldg(pr.grec + 3 * j);
      const float vx = gi.U[0] - uj.x, vy = gi.U[1] - uj.y, vz = gi.U[2] - uj.z;
      const RotV R = rot_apply_cs(gi.cs[0], gi.cs[1], gi.cs[2], gi.cs[3], gi.cs[4], gi.cs[5], vx, vy, vz);
      float j0 = sw * (pi[0] - pj[0]), j1 = sw * (pi[1] - pj[1]), j2 = sw * (pi[2] - pj[2]);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        j0 -= sw * R.g[m][0] * pi[3 + m];
        j1 -= sw * R.g[m][1] * pi[3 + m];
        j2 -= sw * R.g[m][2] * pi[3 + m];
      }
      q[0] += sw * j0; q[1] += sw * j1; q[2] += sw * j2;
#pragma unroll
      for (int m = 0; m < 3; ++m) q[3 + m] -= sw * (R.g[m][0] * j0 + R.g[m][1] * j1 + R.g[m][2] * j2);
    };
    auto in_edge = [&](int j) {
      float pj[6];
      load_vec(pr.vrec, j, pj);
      const GeoRec gj = load_geo(pr.grec, j);
      const float vx = gj.U[0] - gi.U[0], vy = gj.U[1] - gi.U[1], vz = gj.U[2] - gi.U[2];
      const RotV R = rot_apply_cs(gj.cs[0], gj.cs[1], gj.cs[2], gj.cs[3], gj.cs[4], gj.cs[5], vx, vy, vz);
      float j0 = sw * (pj[0] - pi[0]), j1 = sw * (pj[1] - pi[1]), j2 = sw * (pj[2] - pi[2]);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        j0 -= sw * R.g[m][0] * pj[3 + m];
        j1 -= sw * R.g[m][1] * pj[3 + m];
        j2 -= sw * R.g[m][2] * pj[3 + m];
      }
      q[0] -= sw * j0; q[1] -= sw * j1; q[2] -= sw * j2;
    };
    if (G3) {
      const Stencil3 st = stencil3(pr, i);
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (st.ok[t]) own_edge(i + st.off[t]);
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (st.ok[t]) in_edge(i + st.off[t]);
    } else {
#pragma unroll
      for (int t = 0; t < KB + 1; ++t) {
        // t < KB: one prefetched out-edge (if the row has it); t == KB: the rest of a longer row
        const int kb = t < KB ? o0 + t : o0 + KB, ke = t < KB ? min(o0 + t + 1, o1) : o1;
        for (int k = kb; k < ke; ++k) own_edge(t < KB ? jo[t] : pr.e1[k]);
      }
#pragma unroll
      for (int t = 0; t < KB + 1; ++t) {
        const int kb = t < KB ? n0 + t : n0 + KB, ke = t < KB ? min(n0 + t + 1, n1) : n1;
        for (int k = kb; k < ke; ++k) in_edge(t < KB ? ji[t] : pr.isrc[k]);
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
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

// ---------------------------------------------------------------------------
// PCGStep: applyJTJ fused with the direction update, ARAP mesh (tiled)
// ---------------------------------------------------------------------------
// One block per vertex tile of VT vertices (the tile-chunk table), one vertex
// per thread.  The block stages the tile's vertices and its halo (the
// out-of-tile neighbours, a table built at planning) in shared memory: the
// displacement rows of the direction p = M^-1 r + beta p_old (formed here,
// halo included, with the same roundings everywhere) and the rest position U.
// With M_i = sum_m p_i,m dR/dA_m(A_i) formed once per vertex (rot3 /
// rot3_dir), the linearized residual of an out-edge e = (i, j) is
//   t_e = J_e p = s_w [(p_i,d - p_j,d) - M_i v],   v = U_i - U_j;
// it adds s_w t_e to i's displacement rows and its angle rows
// -s_w (dR/dA_m v) . t_e are summed through S_i = sum_e t_e v^T, one
// contraction per vertex (rot3_contract) instead of three derivative vectors
// per edge.  Each t_e goes to a shared-memory slot; in-edges that start
// outside the tile are evaluated edge-parallel from their source's data into
// further slots; every vertex then subtracts s_w t_e of its in-edges, read
// from their slots (a slot table built at planning).  So each residual is
// evaluated once inside a tile and once more per tile border it crosses, no
// atomic is used, and every row is summed in a fixed order.

// Rotation R = Rz(az) Ry(ay) Rx(ax) from the angles' cos / sin, with
// u' = dR_:0 / day; the angle derivatives are then
//   dR/dax = [0 | R_:2 | -R_:1],  dR/day = [u' | sin ax R_:0 | cos ax R_:0],
//   dR/daz = rows (-R_1:, R_0:, 0).
struct Rot3 {
  float r[3][3];
  float ud[3];
  float ca, sa;
};
__device__ __forceinline__ Rot3 rot3(const float cs[6]) {
  const float ca = cs[0], sa = cs[1], cb = cs[2], sb = cs[3], cc = cs[4], sc = cs[5];
  const float a1 = sa * sb, a2 = ca * sb;
  Rot3 o;
  o.r[0][0] = cb * cc; o.r[0][1] = fmaf(a1, cc, -ca * sc); o.r[0][2] = fmaf(a2, cc, sa * sc);
  o.r[1][0] = cb * sc; o.r[1][1] = fmaf(a1, sc, ca * cc);  o.r[1][2] = fmaf(a2, sc, -sa * cc);
  o.r[2][0] = -sb;     o.r[2][1] = sa * cb;                o.r[2][2] = ca * cb;
  o.ud[0] = -sb * cc; o.ud[1] = -sb * sc; o.ud[2] = -cb;
  o.ca = ca; o.sa = sa;
  return o;
}
// M = pa dR/dax + pb dR/day + pc dR/daz
__device__ __forceinline__ void rot3_dir(const Rot3& R, float pa, float pb, float pc, float (&M)[3][3]) {
  const float dz[3][3] = {{-R.r[1][0], -R.r[1][1], -R.r[1][2]}, {R.r[0][0], R.r[0][1], R.r[0][2]}, {0.f, 0.f, 0.f}};
  const float bs = pb * R.sa, bc = pb * R.ca;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    M[i][0] = fmaf(pb, R.ud[i], pc * dz[i][0]);
    M[i][1] = fmaf(pa, R.r[i][2], fmaf(bs, R.r[i][0], pc * dz[i][1]));
    M[i][2] = fmaf(-pa, R.r[i][1], fmaf(bc, R.r[i][0], pc * dz[i][2]));
  }
}
// (<dR/dax, S>, <dR/day, S>, <dR/daz, S>), <A, B> = sum_ij A_ij B_ij
__device__ __forceinline__ void rot3_contract(const Rot3& R, const float (&S)[3][3], float (&o)[3]) {
  float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a = fmaf(R.r[i][2], S[i][1], fmaf(-R.r[i][1], S[i][2], a));
    b = fmaf(R.ud[i], S[i][0], fmaf(R.r[i][0], fmaf(R.sa, S[i][1], R.ca * S[i][2]), b));
    c = fmaf(-R.r[1][i], S[0][i], fmaf(R.r[0][i], S[1][i], c));
  }
  o[0] = a; o[1] = b; o[2] = c;
}

// The direction of vertex v, components [0, NC): p = M^-1 r + beta p_old
// (update) or the given p; the same roundings wherever it is formed.
template <int NC>
__device__ __forceinline__ void mesh_direction(const MeshProb& pr, int v, long long pl, int update, float beta,
                                               const float* __restrict__ pin, float (&o)[NC]) {
  if (update) {
    float m[NC < 4 ? 1 : 4];
#pragma unroll
    for (int k = 0; k < (NC < 4 ? 1 : 4); ++k) m[k] = __ldg(pr.m + k * pl + v);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      o[c] = __fmul_rn(m[c < 3 ? 0 : c - 2], pr.r[c * pl + v]);
      if (beta != 0.0f) o[c] = __fmaf_rn(beta, pin[c * pl + v], o[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) o[c] = pin[c * pl + v];
  }
}

// J_e p of an edge (a, b) from a's matrix M_a: s_w [(p_a - p_b) - M_a v], v = U_a - U_b
__device__ __forceinline__ void edge_jp(float sw, const float (&M)[3][3], const float* pa, const float* pb,
                                        const float (&v)[3], float (&t)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float mv = fmaf(M[a][0], v[0], fmaf(M[a][1], v[1], M[a][2] * v[2]));
    t[a] = sw * ((pa[a] - pb[a]) - mv);
  }
}

#ifndef MESH_TILED_MIN_BLOCKS
#define MESH_TILED_MIN_BLOCKS 4   // resident blocks per SM the tiled apply is compiled for
#endif

__global__ void __launch_bounds__(NT, MESH_TILED_MIN_BLOCKS) k_mesh_apply_tiled(
    const MeshProb* __restrict__ probs, const Chunk* __restrict__ tchunks, double* __restrict__ part,
    const float* __restrict__ p_override, int par, int update) {
  pdl_begin();
  const Chunk ch = tchunks[blockIdx.x];
  const MeshProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  __shared__ float spu[6][VT + MT_HALO];   // the tile's vertices, then its halo: p_d (3), U (3)
  __shared__ float st[3][MT_SLOTS];        // J_e p of the tile's out-edges, then of the remote in-edges
  const long long pl = pr.Vp;
  const float sw = pr.s_w;
  const float beta = s->beta_f;
  const float* __restrict__ pin = p_override ? p_override : pr.p + (long long)(par & 1) * 6 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 6 * pl;
  const int tid = threadIdx.x;
  const int vb = ch.begin, ve = ch.end, T = vb / VT;
  const int i = vb + tid;
  const bool own = i < ve;
  const int ebase = pr.orow[vb], nout = pr.orow[ve] - ebase;
  const int ibase = pr.irow[vb];
  // A: this vertex's direction and geometry, its edge tables fetched ahead
  int o0 = 0, o1 = 0, n0 = 0, n1 = 0;
  int ln[KB], sl[KB];
  float pi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float ui[3] = {0.f, 0.f, 0.f}, cs[6] = {1.f, 0.f, 1.f, 0.f, 1.f, 0.f};
  if (own) {
    o0 = pr.orow[i]; o1 = pr.orow[i + 1];
    n0 = pr.irow[i]; n1 = pr.irow[i + 1];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      ln[t] = o0 + t < o1 ? pr.lnbr[o0 + t] : 0;
      sl[t] = n0 + t < n1 ? pr.itslot[n0 + t] : 0;
    }
    mesh_direction<6>(pr, i, pl, update, beta, pin, pi);
    if (update) {
#pragma unroll
      for (int c = 0; c < 6; ++c) pout[c * pl + i] = pi[c];
    }
    const GeoRec g = load_geo(pr.grec, i);
#pragma unroll
    for (int c = 0; c < 3; ++c) ui[c] = g.U[c];
#pragma unroll
    for (int c = 0; c < 6; ++c) cs[c] = g.cs[c];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) { spu[c][tid] = pi[c]; spu[3 + c][tid] = ui[c]; }
  {
    const int h0 = pr.hptr[T], nh = pr.hptr[T + 1] - h0;
    for (int l = tid; l < nh; l += NT) {
      const int j = pr.hvtx[h0 + l];
      float pj[3];
      mesh_direction<3>(pr, j, pl, update, beta, pin, pj);
      const float4 g = __ldg(pr.grec + 3 * j);
      spu[0][VT + l] = pj[0]; spu[1][VT + l] = pj[1]; spu[2][VT + l] = pj[2];
      spu[3][VT + l] = g.x; spu[4][VT + l] = g.y; spu[5][VT + l] = g.z;
    }
  }
  __syncthreads();
  // B: own edges (displacement rows, S_i), their J_e p into the slots
  float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float S[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (own) {
    float M[3][3];
    rot3_dir(rot3(cs), pi[3], pi[4], pi[5], M);
    auto own_edge = [&](int k, int l) {
      const float pj[3] = {spu[0][l], spu[1][l], spu[2][l]};
      const float v[3] = {ui[0] - spu[3][l], ui[1] - spu[4][l], ui[2] - spu[5][l]};
      float t[3];
      edge_jp(sw, M, pi, pj, v, t);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        q[a] = fmaf(sw, t[a], q[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) S[a][b] = fmaf(t[a], v[b], S[a][b]);
        st[a][k - ebase] = t[a];
      }
    };
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (o0 + t < o1) own_edge(o0 + t, ln[t]);
    for (int k = o0 + KB; k < o1; ++k) own_edge(k, pr.lnbr[k]);
  }
  {
    // in-edges arriving from outside the tile, edge-parallel, from the source's data
    const int r0 = pr.rptr[T], nr = pr.rptr[T + 1] - r0, h0 = pr.hptr[T];
    for (int r = tid; r < nr; r += NT) {
      const int w = pr.rin[r0 + r];
      const int dl = w & 0xffff;
      const int j = pr.hvtx[h0 + (w >> 16) - VT];
      float pj[6];
      mesh_direction<6>(pr, j, pl, update, beta, pin, pj);
      const GeoRec gj = load_geo(pr.grec, j);
      float Mj[3][3], t[3];
      rot3_dir(rot3(gj.cs), pj[3], pj[4], pj[5], Mj);
      const float d[3] = {spu[0][dl], spu[1][dl], spu[2][dl]};
      const float v[3] = {gj.U[0] - spu[3][dl], gj.U[1] - spu[4][dl], gj.U[2] - spu[5][dl]};
      edge_jp(sw, Mj, pj, d, v, t);
#pragma unroll
      for (int a = 0; a < 3; ++a) st[a][nout + r] = t[a];
    }
  }
  __syncthreads();
  // C: angle rows, in-edge displacement rows, fit, damping; p.q
  F2 acc = f2_zero();
  if (own) {
    float ga[3];
    rot3_contract(rot3(cs), S, ga);
#pragma unroll
    for (int m = 0; m < 3; ++m) q[3 + m] = -sw * ga[m];
    auto in_edge = [&](int slot) {
#pragma unroll
      for (int a = 0; a < 3; ++a) q[a] = fmaf(-sw, st[a][slot], q[a]);
    };
#pragma unroll
    for (int t = 0; t < KB; ++t)
      if (n0 + t < n1) in_edge(sl[t]);
    for (int k = n0 + KB; k < n1; ++k) in_edge(pr.itslot[k]);
    if (handle_of(pr, i) >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] = fmaf(pr.w_fit, pi[c], q[c]);
    }
    if (pr.lm) {
      const float lam = s->lambda_f;
#pragma unroll
      for (int c = 0; c < 6; ++c) q[c] = fmaf(lam * pr.dc[(c < 3 ? 0 : c - 2) * pl + i], pi[c], q[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      pr.q[c * pl + i] = q[c];
      f2_add_prod(acc, pi[c], q[c]);
    }
  }
  (void)ibase;
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, pr.tchunk_end - pr.tchunk_begin)) {
    double pq, unused;
    gather_partials(part, pr.tchunk_begin, pr.tchunk_end, &s->counter, pq, unused);
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
  F2x2 acc = f2x2_zero();
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
      const float2 r01 = make_float2(rv[c].x, rv[c].y), r23 = make_float2(rv[c].z, rv[c].w);
      f2x2_add_prod(acc, r01, pk_mul(make_float2(m.x, m.y), r01));
      f2x2_add_prod(acc, r23, pk_mul(make_float2(m.z, m.w), r23));
      *reinterpret_cast<float4*>(pr.d + c * pl + v0) = dv[c];
      *reinterpret_cast<float4*>(pr.r + c * pl + v0) = rv[c];
    }
  }
  pdl_trigger();
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc), f2_zero(), &s->counter, pr.vchunk_end - pr.vchunk_begin)) {
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
  F2 e = f2_zero();
  for (int v = ch.begin + threadIdx.x; v < ch.end; v += NT) {
    const int h = handle_of(pr, v);
    if (h < 0) continue;
    float ev = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float dv = pr.x[c * pl + v];
      if (mode == 1) dv += pr.d[c * pl + v];
      const float f = pr.s_f * (dv - pr.htgt[3 * h + c]);
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
  F2 e0 = f2_zero(), e1 = f2_zero();
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
      f2_add(e0, r0 * r0 + r1 * r1 + r2 * r2);
    } else {
      const float ea0 = pr.d[a] - pr.d[b], ea1 = pr.d[pl + a] - pr.d[pl + b];
      const float ea2 = pr.d[2 * pl + a] - pr.d[2 * pl + b];
      const float t3 = pr.d[3 * pl + a], t4 = pr.d[4 * pl + a], t5 = pr.d[5 * pl + a];
      const RotV R2 = rot_apply(pr.x[3 * pl + a] + t3, pr.x[4 * pl + a] + t4, pr.x[5 * pl + a] + t5, vx, vy, vz);
      const float u0 = sw * ((dd0 + ea0) + (vx - R2.rv[0]));
      const float u1 = sw * ((dd1 + ea1) + (vy - R2.rv[1]));
      const float u2 = sw * ((dd2 + ea2) + (vz - R2.rv[2]));
      f2_add(e0, u0 * u0 + u1 * u1 + u2 * u2);
      const float l0 = r0 + sw * ea0 - sw * (R.g[0][0] * t3 + R.g[1][0] * t4 + R.g[2][0] * t5);
      const float l1 = r1 + sw * ea1 - sw * (R.g[0][1] * t3 + R.g[1][1] * t4 + R.g[2][1] * t5);
      const float l2 = r2 + sw * ea2 - sw * (R.g[0][2] * t3 + R.g[1][2] * t4 + R.g[2][2] * t5);
      f2_add(e1, l0 * l0 + l1 * l1 + l2 * l2);
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
  if (L.dim == 2) return launch_wg_init(L, k_outer, dmin, dmax);
  if (L.dim == 12) return launch_ed_init(L, k_outer, dmin, dmax);
  launch_pdl(k_mesh_init_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks);
  if (L.grid3)
    launch_pdl(k_mesh_init_pull<true>, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, k_outer, dmin, dmax);
  else
    launch_pdl(k_mesh_init_pull<false>, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, k_outer, dmin,
               dmax);
}

void launch_mesh_apply(const MeshLaunch& L, const float* p_override, int par, int update) {
  if (L.dim == 2) return launch_wg_apply(L, p_override, par, update);
  if (L.dim == 12) return launch_ed_apply(L, p_override, par, update);
  if (!L.grid3 && L.tchunks) {
    launch_pdl(k_mesh_apply_tiled, L.ntchunks, NT, 0, L.stream, L.probs, L.tchunks, L.part, p_override, par, update);
    return;
  }
  launch_pdl(k_mesh_apply_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, p_override, par, update);
  if (L.grid3)
    launch_pdl(k_mesh_apply_pull<true>, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part);
  else
    launch_pdl(k_mesh_apply_pull<false>, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part);
}

void launch_mesh_update(const MeshLaunch& L, int par) {
  if (L.dim == 2) return launch_wg_update(L, par);
  if (L.dim == 12) return launch_ed_update(L, par);
  launch_pdl(k_mesh_update, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, par);
}

void launch_mesh_energy(const MeshLaunch& L, int mode, int hist_idx) {
  if (L.dim == 2) return launch_wg_energy(L, mode, hist_idx);
  if (L.dim == 12) return launch_ed_energy(L, mode, hist_idx);
  launch_pdl(k_mesh_energy_v, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, L.part, mode);
  launch_pdl(k_mesh_energy_e, L.nechunks, NT, 0, L.stream, L.probs, L.echunks, L.part, mode, hist_idx);
}

void launch_mesh_step(const MeshLaunch& L, int cond) {
  if (L.dim == 2) return launch_wg_step(L, cond);
  if (L.dim == 12) return launch_ed_step(L, cond);
  launch_pdl(k_mesh_step, L.nvchunks, NT, 0, L.stream, L.probs, L.vchunks, cond);
}

}  // namespace optgb
