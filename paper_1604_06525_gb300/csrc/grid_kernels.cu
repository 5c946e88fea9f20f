// Matrix-free grid kernels (Sec. 4.1 "Stencil-based Array Access").
//
// One block per chunk of 32x8 tiles.  Each tile is staged with a one-pixel
// halo in shared memory (the 5-point stencil of Fig. 24 / Fig. 27), then one
// thread computes the output rows of one pixel in gather form: the residuals
// centred at the pixel ("own") and the residuals of the four neighbours that
// reach it ("incoming") -- the set the paper's stencil JTJ generator finds by
// shifting the residual template (Sec. 5.3.1, Fig. 10).
//
//   k_grid_init   PCGInit: F, b = -J^T F, diag(J^T J), M^-1, r = b, p = z = M^-1 r,
//                 delta = 0, float64 r.z and E                     (Sec. 4.2 evalJTF)
//   k_grid_apply  PCGStep1: p = z + beta p (from r, M^-1, p_old, halo included),
//                 q = (J^T J + lambda D) p, float64 p.q -> alpha   (Sec. 4.2 applyJTJ)
//   k_grid_update PCGStep2: delta += alpha p, r -= alpha q, z = M^-1 r, float64 r.z -> beta
//   k_grid_energy E(x) (evalF) or, for LM, E(x + delta) and |F(x) + J(x) delta|^2
//   k_grid_step   x += delta (GN always, LM when the step was accepted)
//
// ARAP warp algebra (unknown displacement d = O - U, v = U_k - U_{k+d}):
//   r_{k,d}  = s_w [(d_k - d_{k+d}) + (v - R(t_k) v)]                  (= Fig. 24)
//   dr/dd_k  = s_w I,  dr/dd_{k+d} = -s_w I,  dr/dt_k = -s_w R'(t_k) v,
//   R'(t) v  = (-sin t v.x - cos t v.y, cos t v.x - sin t v.y).
// Poisson algebra (per channel): r_{k,d} = (X_k - X_{k+d}) - (T_k - T_{k+d});
//   the residual of a free neighbour towards k is exactly -r_{k,d}.
#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

// stencil directions (+x, -x, +y, -y) of Fig. 24 / Fig. 27
__device__ __forceinline__ int dx4(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
__device__ __forceinline__ int dy4(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }

__device__ __forceinline__ int tile_x0(int tc) { return (tc & 0xffff) * TW; }
__device__ __forceinline__ int tile_y0(int tc) { return (tc >> 16) * TH; }
__device__ __forceinline__ int tile_id(const GridProb& pr, int tc) {
  return (tc >> 16) * pr.ntx + (tc & 0xffff);
}

// ---------------------------------------------------------------------------
// ARAP image warping
// ---------------------------------------------------------------------------
struct WarpStage {
  float a[HH][HW];     // dx  (init / energy) or p.x (apply)
  float b[HH][HW];     // dy  or p.y
  float t[HH][HW];     // theta (energy) or p.theta (apply)
  float cs[HH][HW];    // cos theta
  float sn[HH][HW];    // sin theta
  float ux[HH][HW];
  float uy[HH][HW];
  float ea[HH][HW];    // energy trial: delta x / delta y / delta theta
  float eb[HH][HW];
  float et[HH][HW];
  unsigned char v[HH][HW];
};

__global__ void __launch_bounds__(NT) k_warp_init(const GridProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  const int* __restrict__ tiles,
                                                  double* __restrict__ part, int k_outer,
                                                  float dmin, float dmax) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  __shared__ WarpStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float sw = pr.s_w, sf = pr.s_f, wreg = pr.w_reg, wfit = pr.w_fit;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc_rz = 0.f, acc_E = 0.f;
  for (int t = ch.begin; t < ch.end; ++t) {
    const int tc = tiles[t];
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    for (int hc = threadIdx.x; hc < HW * HH; hc += NT) {
      const int hy = hc / HW, hx = hc - hy * HW;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      float dx = 0.f, dy = 0.f, th = 0.f, ux = 0.f, uy = 0.f;
      unsigned char v = 0;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const long long i = (long long)gy * P + gx;
        dx = pr.x[i];
        dy = pr.x[pl + i];
        th = pr.x[2 * pl + i];
        ux = pr.c[i];
        uy = pr.c[pl + i];
        v = pr.mask ? (pr.mask[i] == 0) : 1;
      }
      float sn, cs;
      sincosf(th, &sn, &cs);
      st.a[hy][hx] = dx; st.b[hy][hx] = dy; st.cs[hy][hx] = cs; st.sn[hy][hx] = sn;
      st.ux[hy][hx] = ux; st.uy[hy][hx] = uy; st.v[hy][hx] = v;
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < W && gy < H) {
      const int lx = tx + 1, ly = ty + 1;
      const long long i = (long long)gy * P + gx;
      const float dxi = st.a[ly][lx], dyi = st.b[ly][lx];
      const float ci = st.cs[ly][lx], si = st.sn[ly][lx];
      const float uxi = st.ux[ly][lx], uyi = st.uy[ly][lx];
      float gdx = 0.f, gdy = 0.f, gt = 0.f, diag_d = 0.f, diag_t = 0.f, e = 0.f;
      if (st.v[ly][lx]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int nx = lx + dx4(k), ny = ly + dy4(k);
          if (!st.v[ny][nx]) continue;
          const float vx = uxi - st.ux[ny][nx], vy = uyi - st.uy[ny][nx];
          const float ddx = dxi - st.a[ny][nx], ddy = dyi - st.b[ny][nx];
          // own residual (centre i, rotation theta_i)
          const float rx = sw * (ddx + (vx - (ci * vx - si * vy)));
          const float ry = sw * (ddy + (vy - (si * vx + ci * vy)));
          const float jx = -sw * (-si * vx - ci * vy);   // dr/dtheta_i
          const float jy = -sw * (ci * vx - si * vy);
          gdx += sw * rx;
          gdy += sw * ry;
          gt += jx * rx + jy * ry;
          diag_t += jx * jx + jy * jy;
          e += rx * rx + ry * ry;
          // incoming residual (centre j, rotation theta_j, v' = -v)
          const float cj = st.cs[ny][nx], sj = st.sn[ny][nx];
          const float r2x = sw * (-ddx + (-vx - (cj * -vx - sj * -vy)));
          const float r2y = sw * (-ddy + (-vy - (sj * -vx + cj * -vy)));
          gdx -= sw * r2x;
          gdy -= sw * r2y;
          diag_d += 2.0f * wreg;
        }
        const int tid = tile_id(pr, tc);
        for (int h = pr.hbeg[tid]; h < pr.hbeg[tid + 1]; ++h) {
          if (pr.hpix[h] == (int)i) {
            const float fx = sf * (dxi - pr.htgt[2 * h]);
            const float fy = sf * (dyi - pr.htgt[2 * h + 1]);
            gdx += sf * fx;
            gdy += sf * fy;
            diag_d += wfit;
            e += fx * fx + fy * fy;
          }
        }
      }
      float dcd, dct;
      const float md = minv_entry(diag_d, lam, dmin, dmax, pr.use_precond, &dcd);
      const float mt = minv_entry(diag_t, lam, dmin, dmax, pr.use_precond, &dct);
      const float bx = -gdx, by = -gdy, bt = -gt;
      pr.r[i] = bx; pr.r[pl + i] = by; pr.r[2 * pl + i] = bt;
      pr.m[i] = md; pr.m[pl + i] = mt;
      pr.d[i] = 0.f; pr.d[pl + i] = 0.f; pr.d[2 * pl + i] = 0.f;
      if (pr.lm) { pr.dc[i] = dcd; pr.dc[pl + i] = dct; }
      if (pr.jtf_out) { pr.jtf_out[i] = gdx; pr.jtf_out[pl + i] = gdy; pr.jtf_out[2 * pl + i] = gt; }
      if (pr.diag_out) { pr.diag_out[i] = diag_d; pr.diag_out[pl + i] = diag_t; }
      acc_rz += md * (bx * bx + by * by) + mt * bt * bt;
      acc_E += e;
    }
    __syncthreads();
  }
  if (publish_partials(part, blockIdx.x, acc_rz, acc_E, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double rz, E;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, rz, E);
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

// Cells of the one-pixel halo ring around a 32x8 tile: 2*HW + 2*TH = 84.
constexpr int NHALO = 2 * HW + 2 * TH;

__device__ __forceinline__ void halo_cell(int h, int& hy, int& hx) {
  if (h < HW) { hy = 0; hx = h; }
  else if (h < 2 * HW) { hy = HH - 1; hx = h - HW; }
  else if (h < 2 * HW + TH) { hy = h - 2 * HW + 1; hx = 0; }
  else { hy = h - 2 * HW - TH + 1; hx = HW - 1; }
}

// Global values of one staged warp cell, held in registers between the load
// (issued one tile ahead) and the shared-memory store.
struct WarpCell {
  float r0, r1, r2, m0, m1, p0, p1, p2, th, u0, u1;
  int inb;
  int v;
};

__device__ __forceinline__ void warp_cell_load(WarpCell& c, const GridProb& pr, const float* __restrict__ pin,
                                               int gx, int gy, int update, int use_beta) {
  c.r0 = c.r1 = c.r2 = c.m0 = c.m1 = c.p0 = c.p1 = c.p2 = c.th = c.u0 = c.u1 = 0.f;
  c.v = 0;
  c.inb = (gx >= 0 && gx < pr.W && gy >= 0 && gy < pr.H);
  if (!c.inb) return;
  const long long pl = pr.plane;
  const long long i = (long long)gy * pr.P + gx;
  if (update) {
    c.r0 = __ldg(pr.r + i);
    c.r1 = __ldg(pr.r + pl + i);
    c.r2 = __ldg(pr.r + 2 * pl + i);
    c.m0 = __ldg(pr.m + i);
    c.m1 = __ldg(pr.m + pl + i);
  }
  if (!update || use_beta) {
    c.p0 = __ldg(pin + i);
    c.p1 = __ldg(pin + pl + i);
    c.p2 = __ldg(pin + 2 * pl + i);
  }
  c.th = __ldg(pr.x + 2 * pl + i);
  c.u0 = __ldg(pr.c + i);
  c.u1 = __ldg(pr.c + pl + i);
  c.v = pr.mask ? (__ldg(pr.mask + i) == 0) : 1;
}

struct WarpApplyStage {
  float a[HH][HW], b[HH][HW], t[HH][HW];   // direction p (x, y, theta)
  float cs[HH][HW], sn[HH][HW];            // cos / sin theta
  float ux[HH][HW], uy[HH][HW];            // UrShape
  unsigned char v[HH][HW];                 // residuals touching the cell are valid
};

// Direction p = M^-1 r + beta p_old (or the caller's p) and trig of theta
// into shared memory; owned cells also write the new direction.
__device__ __forceinline__ void warp_cell_store(WarpApplyStage& st, int hy, int hx, const WarpCell& c,
                                                int update, int use_beta, float beta,
                                                float* __restrict__ pout, const GridProb& pr,
                                                long long i_owned) {
  float px = 0.f, py = 0.f, pt = 0.f, cs = 1.f, sn = 0.f;
  if (c.inb) {
    if (update) {
      px = c.m0 * c.r0;
      py = c.m0 * c.r1;
      pt = c.m1 * c.r2;
      if (use_beta) {
        px += beta * c.p0;
        py += beta * c.p1;
        pt += beta * c.p2;
      }
      if (i_owned >= 0) {
        const long long pl = pr.plane;
        pout[i_owned] = px;
        pout[pl + i_owned] = py;
        pout[2 * pl + i_owned] = pt;
      }
    } else {
      px = c.p0; py = c.p1; pt = c.p2;
    }
    sincosf(c.th, &sn, &cs);
  }
  st.a[hy][hx] = px; st.b[hy][hx] = py; st.t[hy][hx] = pt;
  st.cs[hy][hx] = cs; st.sn[hy][hx] = sn;
  st.ux[hy][hx] = c.u0; st.uy[hy][hx] = c.u1;
  st.v[hy][hx] = (unsigned char)c.v;
}

// q = (J^T J + lambda D) p for the warp; with `update` the direction is
// first advanced, p = M^-1 r + beta p_old, for every staged pixel (halo
// included) and written for the owned pixels.  The global loads of tile t+1
// are issued before tile t is computed, so they are in flight meanwhile.
__global__ void __launch_bounds__(NT, 3) k_warp_apply(const GridProb* __restrict__ probs,
                                                      const Chunk* __restrict__ chunks,
                                                      const int* __restrict__ tiles,
                                                      double* __restrict__ part,
                                                      const float* __restrict__ p_in_override,
                                                      int par, int update) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  __shared__ WarpApplyStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float sw = pr.s_w, wfit = pr.w_fit;
  const float beta = s->beta_f;
  const int use_beta = beta != 0.0f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const float* __restrict__ pin = p_in_override ? p_in_override : pr.p + (long long)(par & 1) * 3 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 3 * pl;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const bool has_halo = tid < NHALO;
  int hhy = 0, hhx = 0;
  if (has_halo) halo_cell(tid, hhy, hhx);
  float acc = 0.f;
  WarpCell A, B;
  int tc = tiles[ch.begin];
  warp_cell_load(A, pr, pin, tile_x0(tc) + tx, tile_y0(tc) + ty, update, use_beta);
  if (has_halo) warp_cell_load(B, pr, pin, tile_x0(tc) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    const int gx = x0 + tx, gy = y0 + ty;
    const long long i = (long long)gy * P + gx;
    __syncthreads();
    warp_cell_store(st, ty + 1, tx + 1, A, update, use_beta, beta, pout, pr, (gx < W && gy < H) ? i : -1);
    if (has_halo) warp_cell_store(st, hhy, hhx, B, update, use_beta, beta, pout, pr, -1);
    __syncthreads();
    const int tcur = tc;
    if (t + 1 < ch.end) {
      tc = tiles[t + 1];
      warp_cell_load(A, pr, pin, tile_x0(tc) + tx, tile_y0(tc) + ty, update, use_beta);
      if (has_halo) warp_cell_load(B, pr, pin, tile_x0(tc) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
    }
    if (gx < W && gy < H) {
      const int lx = tx + 1, ly = ty + 1;
      const float pxi = st.a[ly][lx], pyi = st.b[ly][lx], pti = st.t[ly][lx];
      float qx = 0.f, qy = 0.f, qt = 0.f;
      if (st.v[ly][lx]) {
        const float ci = st.cs[ly][lx], si = st.sn[ly][lx];
        const float uxi = st.ux[ly][lx], uyi = st.uy[ly][lx];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int nx = lx + dx4(k), ny = ly + dy4(k);
          if (!st.v[ny][nx]) continue;
          const float vx = uxi - st.ux[ny][nx], vy = uyi - st.uy[ny][nx];
          const float pxj = st.a[ny][nx], pyj = st.b[ny][nx], ptj = st.t[ny][nx];
          // own residual row: J p = s_w[(p_i - p_j) - R'(t_i) v p_t,i]
          const float gx_ = -sw * (-si * vx - ci * vy);   // dr/dtheta_i
          const float gy_ = -sw * (ci * vx - si * vy);
          const float jpx = sw * (pxi - pxj) + gx_ * pti;
          const float jpy = sw * (pyi - pyj) + gy_ * pti;
          qx += sw * jpx;
          qy += sw * jpy;
          qt += gx_ * jpx + gy_ * jpy;
          // incoming residual row (centre j, v' = -v): d/dd_i = -s_w I
          const float cj = st.cs[ny][nx], sj = st.sn[ny][nx];
          const float hx_ = -sw * (-sj * -vx - cj * -vy);
          const float hy_ = -sw * (cj * -vx - sj * -vy);
          const float kpx = sw * (pxj - pxi) + hx_ * ptj;
          const float kpy = sw * (pyj - pyi) + hy_ * ptj;
          qx -= sw * kpx;
          qy -= sw * kpy;
        }
        const int tid_ = tile_id(pr, tcur);
        for (int h = pr.hbeg[tid_]; h < pr.hbeg[tid_ + 1]; ++h) {
          if (pr.hpix[h] == (int)i) { qx += wfit * pxi; qy += wfit * pyi; }
        }
        if (pr.lm) {
          const float dd = pr.dc[i], dt = pr.dc[pl + i];
          qx += lam * dd * pxi;
          qy += lam * dd * pyi;
          qt += lam * dt * pti;
        }
      }
      pr.q[i] = qx; pr.q[pl + i] = qy; pr.q[2 * pl + i] = qt;
      acc += pxi * qx + pyi * qy + pti * qt;
    }
  }
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double pq, unused;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, pq, unused);
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

// E(x) (mode 0) or E(x + delta) and |F(x) + J(x) delta|^2 (mode 1).
__global__ void __launch_bounds__(NT) k_warp_energy(const GridProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    const int* __restrict__ tiles,
                                                    double* __restrict__ part, int mode,
                                                    int hist_idx) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  __shared__ WarpStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float sw = pr.s_w, sf = pr.s_f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc0 = 0.f, acc1 = 0.f;
  for (int t = ch.begin; t < ch.end; ++t) {
    const int tc = tiles[t];
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    for (int hc = threadIdx.x; hc < HW * HH; hc += NT) {
      const int hy = hc / HW, hx = hc - hy * HW;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      float dx = 0.f, dy = 0.f, th = 0.f, ux = 0.f, uy = 0.f, ex = 0.f, ey = 0.f, et = 0.f;
      unsigned char v = 0;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const long long i = (long long)gy * P + gx;
        dx = pr.x[i]; dy = pr.x[pl + i]; th = pr.x[2 * pl + i];
        ux = pr.c[i]; uy = pr.c[pl + i];
        if (mode == 1) { ex = pr.d[i]; ey = pr.d[pl + i]; et = pr.d[2 * pl + i]; }
        v = pr.mask ? (pr.mask[i] == 0) : 1;
      }
      float sn, cs;
      sincosf(th, &sn, &cs);
      st.a[hy][hx] = dx; st.b[hy][hx] = dy; st.t[hy][hx] = th;
      st.cs[hy][hx] = cs; st.sn[hy][hx] = sn;
      st.ux[hy][hx] = ux; st.uy[hy][hx] = uy;
      st.ea[hy][hx] = ex; st.eb[hy][hx] = ey; st.et[hy][hx] = et;
      st.v[hy][hx] = v;
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < W && gy < H && st.v[ty + 1][tx + 1]) {
      const int lx = tx + 1, ly = ty + 1;
      const long long i = (long long)gy * P + gx;
      const float dxi = st.a[ly][lx], dyi = st.b[ly][lx];
      const float ci = st.cs[ly][lx], si = st.sn[ly][lx];
      const float uxi = st.ux[ly][lx], uyi = st.uy[ly][lx];
      const float exi = st.ea[ly][lx], eyi = st.eb[ly][lx], eti = st.et[ly][lx];
      float c2 = 0.f, s2 = 0.f;
      if (mode == 1) sincosf(st.t[ly][lx] + eti, &s2, &c2);
      float e0 = 0.f, e1 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nx = lx + dx4(k), ny = ly + dy4(k);
        if (!st.v[ny][nx]) continue;
        const float vx = uxi - st.ux[ny][nx], vy = uyi - st.uy[ny][nx];
        const float ddx = dxi - st.a[ny][nx], ddy = dyi - st.b[ny][nx];
        const float rx = sw * (ddx + (vx - (ci * vx - si * vy)));
        const float ry = sw * (ddy + (vy - (si * vx + ci * vy)));
        if (mode == 0) {
          e0 += rx * rx + ry * ry;
        } else {
          const float edx = exi - st.ea[ny][nx], edy = eyi - st.eb[ny][nx];
          const float tx_ = sw * ((ddx + edx) + (vx - (c2 * vx - s2 * vy)));
          const float ty_ = sw * ((ddy + edy) + (vy - (s2 * vx + c2 * vy)));
          e0 += tx_ * tx_ + ty_ * ty_;
          const float lx_ = rx + sw * edx + (-sw * (-si * vx - ci * vy)) * eti;
          const float ly_ = ry + sw * edy + (-sw * (ci * vx - si * vy)) * eti;
          e1 += lx_ * lx_ + ly_ * ly_;
        }
      }
      const int tid = tile_id(pr, tc);
      for (int h = pr.hbeg[tid]; h < pr.hbeg[tid + 1]; ++h) {
        if (pr.hpix[h] == (int)i) {
          const float fx = sf * (dxi - pr.htgt[2 * h]);
          const float fy = sf * (dyi - pr.htgt[2 * h + 1]);
          if (mode == 0) {
            e0 += fx * fx + fy * fy;
          } else {
            const float gx2 = fx + sf * exi, gy2 = fy + sf * eyi;   // linear in d: trial == model
            e0 += gx2 * gx2 + gy2 * gy2;
            e1 += gx2 * gx2 + gy2 * gy2;
          }
        }
      }
      acc0 += e0;
      acc1 += e1;
    }
    __syncthreads();
  }
  if (publish_partials(part, blockIdx.x, acc0, acc1, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double a, b;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, a, b);
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

// ---------------------------------------------------------------------------
// Poisson image editing (4 channels, constant J)
// ---------------------------------------------------------------------------
struct PoissonStage {
  float x[4][HH][HW];   // X (init / energy) or p (apply)
  float g[4][HH][HW];   // guidance T (init / energy)
  float e[4][HH][HW];   // delta (energy, mode 1)
  unsigned char f[HH][HW];   // 0 = outside, 1 = fixed, 2 = free
};

__device__ __forceinline__ unsigned char poisson_flag(const GridProb& pr, long long i) {
  return pr.mask ? (pr.mask[i] == 0 ? 2 : 1) : 2;
}

__global__ void __launch_bounds__(NT) k_poisson_init(const GridProb* __restrict__ probs,
                                                     const Chunk* __restrict__ chunks,
                                                     const int* __restrict__ tiles,
                                                     double* __restrict__ part, int k_outer,
                                                     float dmin, float dmax) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done) return;
  __shared__ PoissonStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc_rz = 0.f, acc_E = 0.f;
  for (int t = ch.begin; t < ch.end; ++t) {
    const int tc = tiles[t];
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    for (int hc = threadIdx.x; hc < HW * HH; hc += NT) {
      const int hy = hc / HW, hx = hc - hy * HW;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      unsigned char f = 0;
      float xv[4] = {0.f, 0.f, 0.f, 0.f}, gv[4] = {0.f, 0.f, 0.f, 0.f};
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const long long i = (long long)gy * P + gx;
#pragma unroll
        for (int c = 0; c < 4; ++c) { xv[c] = pr.x[c * pl + i]; gv[c] = pr.c[c * pl + i]; }
        f = poisson_flag(pr, i);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) { st.x[c][hy][hx] = xv[c]; st.g[c][hy][hx] = gv[c]; }
      st.f[hy][hx] = f;
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < W && gy < H) {
      const int lx = tx + 1, ly = ty + 1;
      const long long i = (long long)gy * P + gx;
      float gr[4] = {0.f, 0.f, 0.f, 0.f};
      float dg = 0.f, e = 0.f;
      if (st.f[ly][lx] == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int nx = lx + dx4(k), ny = ly + dy4(k);
          const unsigned char fj = st.f[ny][nx];
          if (!fj) continue;
          const float w = fj == 2 ? 2.0f : 1.0f;   // own + (free neighbour) incoming
          dg += w;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float r = (st.x[c][ly][lx] - st.x[c][ny][nx]) - (st.g[c][ly][lx] - st.g[c][ny][nx]);
            gr[c] += w * r;
            e += r * r;
          }
        }
      }
      float dcv;
      const float mv = minv_entry(dg, lam, dmin, dmax, pr.use_precond, &dcv);
      float rz = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float b = -gr[c];
        pr.r[c * pl + i] = b;
        pr.d[c * pl + i] = 0.f;
        if (pr.jtf_out) pr.jtf_out[c * pl + i] = gr[c];
        rz += b * b;
      }
      pr.m[i] = mv;
      if (pr.lm) pr.dc[i] = dcv;
      if (pr.diag_out) pr.diag_out[i] = dg;
      acc_rz += mv * rz;
      acc_E += e;
    }
    __syncthreads();
  }
  if (publish_partials(part, blockIdx.x, acc_rz, acc_E, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double rz, E;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, rz, E);
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

struct PoisCell {
  float r[4], p[4], m;
  int inb;
  int f;
};

__device__ __forceinline__ void pois_cell_load(PoisCell& c, const GridProb& pr, const float* __restrict__ pin,
                                               int gx, int gy, int update, int use_beta) {
#pragma unroll
  for (int k = 0; k < 4; ++k) { c.r[k] = 0.f; c.p[k] = 0.f; }
  c.m = 0.f;
  c.f = 0;
  c.inb = (gx >= 0 && gx < pr.W && gy >= 0 && gy < pr.H);
  if (!c.inb) return;
  const long long pl = pr.plane;
  const long long i = (long long)gy * pr.P + gx;
  if (update) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.r[k] = __ldg(pr.r + k * pl + i);
    c.m = __ldg(pr.m + i);
  }
  if (!update || use_beta) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c.p[k] = __ldg(pin + k * pl + i);
  }
  c.f = pr.mask ? (__ldg(pr.mask + i) == 0 ? 2 : 1) : 2;
}

struct PoisApplyStage {
  float p[4][HH][HW];
  unsigned char f[HH][HW];   // 0 = outside, 1 = fixed, 2 = free
};

__device__ __forceinline__ void pois_cell_store(PoisApplyStage& st, int hy, int hx, const PoisCell& c,
                                                int update, int use_beta, float beta,
                                                float* __restrict__ pout, long long pl, long long i_owned) {
  float pv[4] = {0.f, 0.f, 0.f, 0.f};
  if (c.inb && c.f == 2) {   // fixed pixels carry no unknown: p = 0 there
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pv[k] = update ? c.m * c.r[k] : c.p[k];
      if (update && use_beta) pv[k] += beta * c.p[k];
    }
  }
  if (update && c.inb && i_owned >= 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) pout[k * pl + i_owned] = pv[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) st.p[k][hy][hx] = pv[k];
  st.f[hy][hx] = (unsigned char)(c.inb ? c.f : 0);
}

__global__ void __launch_bounds__(NT, 3) k_poisson_apply(const GridProb* __restrict__ probs,
                                                         const Chunk* __restrict__ chunks,
                                                         const int* __restrict__ tiles,
                                                         double* __restrict__ part,
                                                         const float* __restrict__ p_in_override,
                                                         int par, int update) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  __shared__ PoisApplyStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float beta = s->beta_f;
  const int use_beta = beta != 0.0f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const float* __restrict__ pin = p_in_override ? p_in_override : pr.p + (long long)(par & 1) * 4 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 4 * pl;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const bool has_halo = tid < NHALO;
  int hhy = 0, hhx = 0;
  if (has_halo) halo_cell(tid, hhy, hhx);
  float acc = 0.f;
  PoisCell A, B;
  int tc = tiles[ch.begin];
  pois_cell_load(A, pr, pin, tile_x0(tc) + tx, tile_y0(tc) + ty, update, use_beta);
  if (has_halo) pois_cell_load(B, pr, pin, tile_x0(tc) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    const int gx = x0 + tx, gy = y0 + ty;
    const long long i = (long long)gy * P + gx;
    __syncthreads();
    pois_cell_store(st, ty + 1, tx + 1, A, update, use_beta, beta, pout, pl, (gx < W && gy < H) ? i : -1);
    if (has_halo) pois_cell_store(st, hhy, hhx, B, update, use_beta, beta, pout, pl, -1);
    __syncthreads();
    if (t + 1 < ch.end) {
      tc = tiles[t + 1];
      pois_cell_load(A, pr, pin, tile_x0(tc) + tx, tile_y0(tc) + ty, update, use_beta);
      if (has_halo) pois_cell_load(B, pr, pin, tile_x0(tc) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
    }
    if (gx < W && gy < H) {
      const int lx = tx + 1, ly = ty + 1;
      float q[4] = {0.f, 0.f, 0.f, 0.f};
      if (st.f[ly][lx] == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int nx = lx + dx4(k), ny = ly + dy4(k);
          const unsigned char fj = st.f[ny][nx];
          if (!fj) continue;
          const float w = fj == 2 ? 2.0f : 1.0f;   // own + (free neighbour) incoming
#pragma unroll
          for (int c = 0; c < 4; ++c) q[c] += w * (st.p[c][ly][lx] - st.p[c][ny][nx]);
        }
        if (pr.lm) {
          const float dd = lam * pr.dc[i];
#pragma unroll
          for (int c = 0; c < 4; ++c) q[c] += dd * st.p[c][ly][lx];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pr.q[c * pl + i] = q[c];
        acc += st.p[c][ly][lx] * q[c];
      }
    }
  }
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double pq, unused;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, pq, unused);
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

__global__ void __launch_bounds__(NT) k_poisson_energy(const GridProb* __restrict__ probs,
                                                       const Chunk* __restrict__ chunks,
                                                       const int* __restrict__ tiles,
                                                       double* __restrict__ part, int mode,
                                                       int hist_idx) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  __shared__ PoissonStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc0 = 0.f, acc1 = 0.f;
  for (int t = ch.begin; t < ch.end; ++t) {
    const int tc = tiles[t];
    const int x0 = tile_x0(tc), y0 = tile_y0(tc);
    for (int hc = threadIdx.x; hc < HW * HH; hc += NT) {
      const int hy = hc / HW, hx = hc - hy * HW;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      unsigned char f = 0;
      float xv[4] = {0.f, 0.f, 0.f, 0.f}, gv[4] = {0.f, 0.f, 0.f, 0.f}, ev[4] = {0.f, 0.f, 0.f, 0.f};
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const long long i = (long long)gy * P + gx;
        f = poisson_flag(pr, i);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xv[c] = pr.x[c * pl + i];
          gv[c] = pr.c[c * pl + i];
          if (mode == 1 && f == 2) ev[c] = pr.d[c * pl + i];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) { st.x[c][hy][hx] = xv[c]; st.g[c][hy][hx] = gv[c]; st.e[c][hy][hx] = ev[c]; }
      st.f[hy][hx] = f;
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < W && gy < H && st.f[ty + 1][tx + 1] == 2) {
      const int lx = tx + 1, ly = ty + 1;
      float e0 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nx = lx + dx4(k), ny = ly + dy4(k);
        if (!st.f[ny][nx]) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float r = (st.x[c][ly][lx] - st.x[c][ny][nx]) - (st.g[c][ly][lx] - st.g[c][ny][nx]);
          if (mode == 1) r += st.e[c][ly][lx] - st.e[c][ny][nx];   // linear: trial == model
          e0 += r * r;
        }
      }
      acc0 += e0;
      acc1 += e0;
    }
    __syncthreads();
  }
  if (publish_partials(part, blockIdx.x, acc0, acc1, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double a, b;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, a, b);
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

// ---------------------------------------------------------------------------
// shared grid passes
// ---------------------------------------------------------------------------
// delta += alpha p, r -= alpha q, z = M^-1 r, float64 r.z -> beta.
// Float4 stream over the tile rows (a tile row is 32 floats = 128 B of each
// plane; the pitch keeps rows 16-byte aligned and the pitch padding holds
// zeros in every vector).  All loads of a quad are issued before any use.
template <int NX>
__global__ void __launch_bounds__(NT) k_grid_update(const GridProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    const int* __restrict__ tiles,
                                                    double* __restrict__ part, int par) {
  constexpr int NM = NX == 3 ? 2 : 1;
  constexpr int QPT = TW / 4 * TH;   // float4 quads per tile
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const long long pl4 = pr.plane / 4;
  const int P4 = pr.P / 4;
  const float alpha = s->alpha_f;
  const float4* __restrict__ pn = reinterpret_cast<const float4*>(pr.p + (long long)((par + 1) & 1) * NX * pr.plane);
  const float4* __restrict__ q4 = reinterpret_cast<const float4*>(pr.q);
  const float4* __restrict__ m4 = reinterpret_cast<const float4*>(pr.m);
  float4* __restrict__ d4 = reinterpret_cast<float4*>(pr.d);
  float4* __restrict__ r4 = reinterpret_cast<float4*>(pr.r);
  float acc = 0.f;
  const int nq = (ch.end - ch.begin) * QPT;
  for (int k = threadIdx.x; k < nq; k += NT) {
    const int tc = tiles[ch.begin + k / QPT];
    const int w = k % QPT;
    const int y = tile_y0(tc) + w / (TW / 4);
    if (y >= pr.H) continue;
    const long long j = (long long)y * P4 + tile_x0(tc) / 4 + w % (TW / 4);
    float4 pv[NX], qv[NX], dv[NX], rv[NX], mv[NM];
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      pv[c] = __ldg(pn + c * pl4 + j);
      qv[c] = __ldg(q4 + c * pl4 + j);
      dv[c] = d4[c * pl4 + j];
      rv[c] = r4[c * pl4 + j];
    }
#pragma unroll
    for (int c = 0; c < NM; ++c) mv[c] = __ldg(m4 + c * pl4 + j);
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      // distinct-diagonal plane: warp (x, y) -> 0, theta -> 1; Poisson -> 0
      const float4 m = mv[NX == 3 ? (c == 2 ? 1 : 0) : 0];
      dv[c].x += alpha * pv[c].x; dv[c].y += alpha * pv[c].y;
      dv[c].z += alpha * pv[c].z; dv[c].w += alpha * pv[c].w;
      rv[c].x -= alpha * qv[c].x; rv[c].y -= alpha * qv[c].y;
      rv[c].z -= alpha * qv[c].z; rv[c].w -= alpha * qv[c].w;
      acc += rv[c].x * (m.x * rv[c].x) + rv[c].y * (m.y * rv[c].y) +
             rv[c].z * (m.z * rv[c].z) + rv[c].w * (m.w * rv[c].w);
      d4[c * pl4 + j] = dv[c];
      r4[c * pl4 + j] = rv[c];
    }
  }
  if (publish_partials(part, blockIdx.x, acc, 0.0, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double rz, unused;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, rz, unused);
    if (threadIdx.x == 0) {
      const double beta = rz / s->rz;
      s->beta_f = (float)beta;
      s->rz = rz;
      s->pcg_iters += 1;
      if (rz == 0.0 || !isfinite(rz)) s->pcg_active = 0;
      if (!isfinite(rz)) s->nonfinite = 1;
    }
  }
}

// x += delta over the owned pixels (cond: 0 always, 1 only if s->accept).
template <int NX>
__global__ void __launch_bounds__(NT) k_grid_step(const GridProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  const int* __restrict__ tiles, int cond) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  if (cond && !pr.s->accept) return;
  if (!cond && pr.s->done) return;
  const long long pl = pr.plane;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int t = ch.begin; t < ch.end; ++t) {
    const int tc = tiles[t];
    const int gx = tile_x0(tc) + tx, gy = tile_y0(tc) + ty;
    if (gx >= pr.W || gy >= pr.H) continue;
    const long long i = (long long)gy * pr.P + gx;
#pragma unroll
    for (int c = 0; c < NX; ++c) pr.x[c * pl + i] += pr.d[c * pl + i];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_grid_init(int kind, const GridLaunch& L, int k_outer, float dmin, float dmax) {
  if (kind == K_WARP)
    k_warp_init<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, k_outer, dmin, dmax);
  else
    k_poisson_init<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, k_outer, dmin, dmax);
}

void launch_grid_apply(int kind, const GridLaunch& L, const float* p_override, int par, int update) {
  if (kind == K_WARP)
    k_warp_apply<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, p_override, par, update);
  else
    k_poisson_apply<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, p_override, par, update);
}

void launch_grid_update(int kind, const GridLaunch& L, int par) {
  if (kind == K_WARP)
    k_grid_update<3><<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, par);
  else
    k_grid_update<4><<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, par);
}

void launch_grid_energy(int kind, const GridLaunch& L, int mode, int hist_idx) {
  if (kind == K_WARP)
    k_warp_energy<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, mode, hist_idx);
  else
    k_poisson_energy<<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, L.part, mode, hist_idx);
}

void launch_grid_step(int kind, const GridLaunch& L, int cond) {
  if (kind == K_WARP)
    k_grid_step<3><<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, cond);
  else
    k_grid_step<4><<<L.nchunks, NT, 0, L.stream>>>(L.probs, L.chunks, L.tiles, cond);
}

}  // namespace optgb
