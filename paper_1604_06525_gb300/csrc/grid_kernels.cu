// Matrix-free grid kernels (Sec. 4.1 "Stencil-based Array Access").
//
// One block per chunk of tiles (32 x 8 pixels, or 128 x 8 for grids at least
// 128 pixels wide).  Each tile is staged with a one-pixel halo in shared
// memory (the 5-point stencil of Fig. 24 / Fig. 27), then one thread computes
// the output rows of its pixels in gather form: the residuals centred at the
// pixel ("own") and the residuals of the four neighbours that reach it
// ("incoming") -- the set the paper's stencil JTJ generator finds by shifting
// the residual template (Sec. 5.3.1, Fig. 10).
//
//   PCGInit (Sec. 4.2 evalJTF): F, b = -J^T F, diag(J^T J), M^-1, r = b,
//     delta = 0, float64 r.z and E        k_warp_init(_wide), k_poisson_init(_wide)
//   Two-pass PCG iteration (Sec. 4.1, 4.2):
//     applyJTJ with the direction p = z + beta p_old (halo included),
//     q = (J^T J + lambda D) p, float64 p.q -> alpha
//                                          k_warp_apply(_wide), k_poisson_apply(_wide)
//     vector update delta += alpha p, r -= alpha q, z = M^-1 r, float64 r.z -> beta
//                                          k_grid_update
//   Single-reduction PCG iteration (128-pixel tiles): the update of the
//     previous iteration, the direction, applyJTJ and p.q, q.z, q.M^-1 q, r.z
//     in one launch                        k_warp_fused_wide, k_poisson_fused_wide,
//                                          k_grid_fused_fin (the last step)
//   Energies: E(x) (evalF) or, for LM, E(x + delta) and |F(x) + J(x) delta|^2
//                                          k_warp_energy, k_poisson_energy
//   Outer update: x += delta (GN always, LM when the step was accepted)
//                                          k_grid_step
//
// ARAP warp algebra (unknown displacement d = O - U, v = U_k - U_{k+d}):
//   r_{k,d}  = s_w [(d_k - d_{k+d}) + (v - R(t_k) v)]                  (= Fig. 24)
//   dr/dd_k  = s_w I,  dr/dd_{k+d} = -s_w I,  dr/dt_k = -s_w R'(t_k) v,
//   R'(t) v  = (-sin t v.x - cos t v.y, cos t v.x - sin t v.y).
// Poisson algebra (per channel): r_{k,d} = (X_k - X_{k+d}) - (T_k - T_{k+d});
//   the residual of a free neighbour towards k is exactly -r_{k,d}.
#include <mutex>

#include "opt_internal.cuh"
#include "opt_launch.h"

namespace optgb {

namespace {

// stencil directions (+x, -x, +y, -y) of Fig. 24 / Fig. 27
__device__ __forceinline__ int dx4(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
__device__ __forceinline__ int dy4(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }

__device__ __forceinline__ int tile_x0(int tc, int tw) { return (tc & 0xffff) * tw; }
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
  pdl_begin();
  Scalars* s = pr.s;
  if (s->done) return;
  __shared__ WarpStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float sw = pr.s_w, sf = pr.s_f, wreg = pr.w_reg, wfit = pr.w_fit;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  F2 acc_rz = f2_zero(), acc_E = f2_zero();
  const int nsub = pr.tw / TW;
  for (int ts = ch.begin * nsub; ts < ch.end * nsub; ++ts) {
    const int tc = tiles[ts / nsub];
    const int x0 = tile_x0(tc, pr.tw) + TW * (ts % nsub), y0 = tile_y0(tc);
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
      if (pr.csn) { pr.csn[i] = ci; pr.csn[pl + i] = si; }
      if (pr.jtf_out) { pr.jtf_out[i] = gdx; pr.jtf_out[pl + i] = gdy; pr.jtf_out[2 * pl + i] = gt; }
      if (pr.diag_out) { pr.diag_out[i] = diag_d; pr.diag_out[pl + i] = diag_t; }
      f2_add_prod(acc_rz, bx, __fmul_rn(md, bx));
      f2_add_prod(acc_rz, by, __fmul_rn(md, by));
      f2_add_prod(acc_rz, bt, __fmul_rn(mt, bt));
      f2_add(acc_E, e);
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
  pdl_begin();
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
  F2 acc = f2_zero();
  WarpCell A, B;
  int tc = tiles[ch.begin];
  warp_cell_load(A, pr, pin, tile_x0(tc, 32) + tx, tile_y0(tc) + ty, update, use_beta);
  if (has_halo) warp_cell_load(B, pr, pin, tile_x0(tc, 32) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, 32), y0 = tile_y0(tc);
    const int gx = x0 + tx, gy = y0 + ty;
    const long long i = (long long)gy * P + gx;
    __syncthreads();
    warp_cell_store(st, ty + 1, tx + 1, A, update, use_beta, beta, pout, pr, (gx < W && gy < H) ? i : -1);
    if (has_halo) warp_cell_store(st, hhy, hhx, B, update, use_beta, beta, pout, pr, -1);
    __syncthreads();
    const int tcur = tc;
    if (t + 1 < ch.end) {
      tc = tiles[t + 1];
      warp_cell_load(A, pr, pin, tile_x0(tc, 32) + tx, tile_y0(tc) + ty, update, use_beta);
      if (has_halo) warp_cell_load(B, pr, pin, tile_x0(tc, 32) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
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
      f2_add_prod(acc, pxi, qx);
      f2_add_prod(acc, pyi, qy);
      f2_add_prod(acc, pti, qt);
    }
  }
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, pr.chunk_end - pr.chunk_begin)) {
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

// ---------------------------------------------------------------------------
// Wide-tile warp apply (tw = 128), staged with asynchronous copies.
// Raw planes of the halo-extended tile (rows y0-1 .. y0+8, columns x0-1 ..
// x0+128) are copied global -> shared with cp.async (16 bytes per thread per
// plane for the quads, 4 bytes for the halo columns), so a whole tile is in
// flight without occupying registers.  Phase 2 turns the raw planes into the
// staged direction p = M^-1 r + beta p_old (and validity bits); once that is
// done the raw buffer is free and the next tile's copies are issued, so they
// overlap phase 3, the stencil (four pixels per thread, horizontal neighbours
// by warp shuffles, vertical neighbours from shared memory).  For every valid
// neighbour pair the own-residual and incoming-residual rows are summed in the
// grouped form
//   q_d,i += w [2 (p_i - p_j) + G_i p_t,i + G_j p_t,j],  q_t,i += w G_i . ((p_i - p_j) + G_i p_t,i)
// with v = U_i - U_j and G_k = -R'(theta_k) v = (s_k v_x + c_k v_y, s_k v_y - c_k v_x).
// ---------------------------------------------------------------------------
constexpr int W4 = 128;          // wide tile width
constexpr int SP = W4 + 8;       // staged row pitch (floats): columns -1..128 live at 3..132
constexpr int SPB = W4 + 32;     // mask row pitch (bytes): columns 0..127 live at 16..143
static_assert(SP == WIDE_BOX_W && SPB == WIDE_BYTE_BOX_W, "staged boxes and tensor-map boxes must agree");
constexpr int NRAW = 12;         // r0 r1 r2 m0 m1 p0 p1 p2 cos sin ux uy
constexpr int NSTG = 8;          // px py pt cos sin ux uy valid, each quad stored as pixels 0 2 1 3

// One staged plane: the halo-extended tile (rows y0 - 1 .. y0 + 8, columns
// x0 - 4 .. x0 + 131 at v[row][0 .. 135]), padded to a multiple of 128 bytes
// so that every plane of a staging area starts where a tensor copy may write.
struct __align__(128) PlaneT {
  float v[HH][SP];
  float pad[16];
};
static_assert(sizeof(PlaneT) % 128 == 0, "plane slots must keep 128-byte alignment");
// The staged byte plane (mask or degree bytes): columns x0 - 16 .. x0 + 143
// at v[row][0 .. 159].
struct __align__(128) BytesT {
  unsigned char v[HH][SPB];
  unsigned char pad[64];
};
static_assert(sizeof(BytesT) % 128 == 0, "byte slots must keep 128-byte alignment");

struct WideSmem {
  PlaneT raw[NRAW];
  float stg[NSTG][HH][SP];       // halo columns -1 / 128 live at 3 / 132, in plain order
  BytesT mk;
  unsigned long long bar;        // tensor-copy completion of the raw planes
};

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float cmp(const float4& a, int k) {
  return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;   // 0: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Tensor copies (TMA) of the staged tiles.  One thread issues one copy per
// plane (box: 136 columns x 10 rows x 1 plane from (x0 - 4, y0 - 1); the byte
// plane: 160 x 10 from (x0 - 16, y0 - 1): both x offsets are multiples of 16
// bytes); the copy engine zero-fills rows and columns outside the tensor, as
// the cp.async path does.  Completion is counted in bytes on an mbarrier in
// shared memory.  Every thread waits for the phase itself, bounded by 1 s of
// %globaltimer: a wait that runs out reports failure (the kernel then sets
// Scalars::timeout and returns; the host reports OPT_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
constexpr unsigned kPlaneBox = HH * SP * 4;     // bytes one plane copy writes
constexpr unsigned kByteBox = HH * SPB;         // bytes one byte-plane copy writes

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Waits for the completion of the phase with the given parity; false once
// limit_ns (1 s) has passed without it.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned long long limit_ns = kBarrierLimitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_plane(PlaneT* dst, const unsigned long long* map, int x, int y, int z,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_bytes(BytesT* dst, const unsigned long long* map, int x, int y,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// tensor copies write only to 128-byte aligned staging areas (checked once
// per launch; an unaligned area is staged by cp.async instead)
__device__ __forceinline__ bool smem_aligned128(const void* p) { return (smem_u32(p) & 127u) == 0u; }
// slab plane index of a plane group (0 r, 1 M^-1, 2 p of parity 0, 3 cos /
// sin, 4 constants)
__device__ __forceinline__ int zslab(const GridProb& pr, int g) { return (pr.zpack >> (6 * g)) & 63; }
// whether a launch stages by tensor copies: the problem has tensor maps and
// the staging area is aligned
__device__ __forceinline__ bool wide_tma(const GridProb& pr, const void* smem) {
  return pr.tmap != nullptr && smem_aligned128(smem);
}
// Kernels that stage only by tensor copies check this first; on failure
// (no tensor maps, or an unaligned staging area, which the 128-byte aligned
// dynamic shared memory rules out) they flag the problem and do nothing.
__device__ __forceinline__ bool tma_ready(const GridProb& pr, const void* smem) {
  if (wide_tma(pr, smem)) return true;
  if (threadIdx.x == 0) atomicExch(&pr.s->misaligned, 1u);
  return false;
}
// tensor map m of a problem (0 slab, 1 unknowns, 2 byte plane)
__device__ __forceinline__ const unsigned long long* tmap_of(const GridProb& pr, int m) { return pr.tmap + 16 * m; }

// Issues the tensor copies of one tile (one thread): raw[k] from the plane
// that plane(k, z, m) names (plane z of map m; z < 0: not copied), the byte
// plane into mk if `bytes`.  Every thread has finished reading the slot
// before the call (a block barrier lies between); the proxy fence orders
// those reads before the copy engine's writes.
template <int NR, class F>
__device__ __forceinline__ void tile_tma(PlaneT* raw, BytesT* mk, F plane, bool bytes, const GridProb& pr, int x0,
                                         int y0, unsigned long long* bar) {
  unsigned total = bytes ? kByteBox : 0u;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    int z, m;
    plane(k, z, m);
    if (z >= 0) total += kPlaneBox;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_expect(bar, total);
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    int z, m;
    plane(k, z, m);
    if (z >= 0) tma_plane(&raw[k], tmap_of(pr, m), x0 - 4, y0 - 1, z, bar);
  }
  if (bytes) tma_bytes(mk, tmap_of(pr, 2), x0 - 16, y0 - 1, bar);
}

// Timeout of a staging wait: flags the problem and returns once the copies
// still in flight into the slot have landed (or another second has passed).
__device__ __forceinline__ void staging_timeout(Scalars* s, unsigned long long* bar, unsigned parity) {
  if (threadIdx.x == 0) {
    atomicExch(&s->timeout, 1u);
    mbar_wait(bar, parity);
  }
}

struct WidePlanes {
  const float* src[NRAW];        // plane base pointers (nullptr: not needed this launch)
};

// Issues the copies of one 128 x 8 tile with its halo into raw[0..NR-1]
// (column x0 + k at 4 + k): quads of the own rows by every thread, of the two
// halo rows by threads 0..63, and the halo columns by threads 64..79 as the
// aligned quad holding column -1 (x0-4 .. x0-1, staged at 0..3) or column
// 128 (x0+128 .. x0+131, staged at 132..135); x0 is a multiple of 128, so
// both quads lie inside the pitched row when valid.  Rows / columns outside
// the grid are zero-filled.  src[k] == nullptr skips plane k.  The bytes of
// the byte plane (mask or degree plane; skipped unless MASK) of the own /
// halo rows land at mk[row][16 + k], those of the halo columns
// as the aligned 4-byte words around them (column -1 at mk[row][15], column
// 128 at mk[row][144]).
template <int NR, bool MASK>
__device__ __forceinline__ void tile_issue(PlaneT* raw, unsigned char (*mk)[SPB],
                                           const float* const* src, const uint8_t* __restrict__ bytes,
                                           const GridProb& pr, int x0, int y0, int tid) {
  const int lane = tid & 31, ty = tid >> 5;
  const int gx = x0 + 4 * lane;
  {
    const int gy = y0 + ty;
    const bool ok = gy < pr.H;
    const long long i = ok ? (long long)gy * pr.P + gx : 0;
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (src[k]) cp_async16(&raw[k].v[ty + 1][4 + 4 * lane], src[k] + i, ok);
    if (MASK) cp_async4(&mk[ty + 1][16 + 4 * lane], bytes + i, ok);
  }
  if (tid < 64) {
    const int row = tid < 32 ? 0 : HH - 1;
    const int gy = y0 - 1 + row;
    const bool ok = gy >= 0 && gy < pr.H;
    const long long i = ok ? (long long)gy * pr.P + gx : 0;
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (src[k]) cp_async16(&raw[k].v[row][4 + 4 * lane], src[k] + i, ok);
    if (MASK) cp_async4(&mk[row][16 + 4 * lane], bytes + i, ok);
  } else if (tid < 64 + 2 * TH) {
    const int h = tid - 64;
    const int row = 1 + (h % TH), side = h / TH;
    const int gy = y0 + row - 1, cx = side ? x0 + W4 : x0 - 4;
    const bool ok = gy < pr.H && (side ? x0 + W4 < pr.W : x0 > 0);
    const long long i = ok ? (long long)gy * pr.P + cx : 0;
    const int col = side ? 4 + W4 : 0;
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (src[k]) cp_async16(&raw[k].v[row][col], src[k] + i, ok);
    if (MASK) cp_async4(&mk[row][side ? 16 + W4 : 12], bytes + i, ok);
  }
  cp_async_commit();
}

// mask byte of the staged halo column (side 0: column -1, side 1: column 128)
__device__ __forceinline__ unsigned char halo_mask(const unsigned char (*mk)[SPB], int row, int side) {
  return mk[row][side ? 16 + W4 : 15];
}

template <bool MASK>
__device__ __forceinline__ void wide_issue(WideSmem& sm, const WidePlanes& pp, const GridProb& pr, int x0, int y0,
                                           int tid) {
  tile_issue<NRAW, MASK>(sm.raw, sm.mk.v, pp.src, pr.mask, pr, x0, y0, tid);
}

// Packed float32 pairs (one instruction for two lanes of a float2).  All are
// correctly rounded IEEE operations, so results do not depend on the packing.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float4 mul4p(const float4& a, const float4& b) {
  return cat4(mul2(lo2(a), lo2(b)), mul2(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 fma4p(float2 a, const float4& x, const float4& y) {
  return cat4(fma2(a, lo2(x), lo2(y)), fma2(a, hi2(x), hi2(y)));
}
// pixel order 0 1 2 3 <-> 0 2 1 3 (its own inverse)
__device__ __forceinline__ float4 swz4(const float4& v) { return make_float4(v.x, v.z, v.y, v.w); }
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }

// Phase 2 for one staged quad: direction, copied geometry and validity (1 / 0),
// stored in the staged order 0 2 1 3 so that pixels {0, 2} and {1, 3} form the
// two float2 packs of the stencil.
template <bool MASK>
__device__ __forceinline__ void wide_stage_quad(WideSmem& sm, int row, int lane, const GridProb& pr, int gx, int gy,
                                                int update, int use_beta, float2 beta2) {
  const int c = 4 + 4 * lane;
  auto R = [&](int k) { return lds4(&sm.raw[k].v[row][c]); };
  float4 a, b, t;
  if (update) {
    const float4 m0 = R(3), m1 = R(4);
    a = mul4p(m0, R(0));
    b = mul4p(m0, R(1));
    t = mul4p(m1, R(2));
    if (use_beta) {
      a = fma4p(beta2, R(5), a);
      b = fma4p(beta2, R(6), b);
      t = fma4p(beta2, R(7), t);
    }
  } else {
    a = R(5); b = R(6); t = R(7);
  }
  sts4(&sm.stg[0][row][c], swz4(a));
  sts4(&sm.stg[1][row][c], swz4(b));
  sts4(&sm.stg[2][row][c], swz4(t));
#pragma unroll
  for (int k = 0; k < 4; ++k) sts4(&sm.stg[3 + k][row][c], swz4(R(8 + k)));
  float vk[4] = {0.f, 0.f, 0.f, 0.f};
  if (gy >= 0 && gy < pr.H) {
    const unsigned int m4 = MASK ? *reinterpret_cast<const unsigned int*>(&sm.mk.v[row][16 + 4 * lane]) : 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      vk[k] = (gx + k < pr.W && (!MASK || ((m4 >> (8 * k)) & 0xffu) == 0u)) ? 1.f : 0.f;
  }
  sts4(&sm.stg[7][row][c], make_float4(vk[0], vk[2], vk[1], vk[3]));
}

// Own values of one float2 pack of pixels.
struct Own2 {
  float2 px, py, pt, c, s, ux, uy;
};

// Adds the grouped own + incoming rows of the pairs (i, j) of one pack (two
// pixels i, each with its neighbour j in the same direction), scaled by the
// validity m_j of the neighbour.  With v = U_i - U_j, a = p_i - p_j and
// G_k = (s_k v_x + c_k v_y, s_k v_y - c_k v_x):
//   q_d,i += m_j [2 a + G_i p_t,i + G_j p_t,j],  q_t,i += m_j G_i . (a + G_i p_t,i).
__device__ __forceinline__ void pair2(const Own2& o, float2 pxj, float2 pyj, float2 ptj, float2 cj, float2 sj,
                                      float2 uxj, float2 uyj, float2 mj, float2& ax, float2& ay, float2& at) {
  const float2 vx = sub2(o.ux, uxj), vy = sub2(o.uy, uyj), nvx = sub2(uxj, o.ux);
  const float2 a = sub2(o.px, pxj), b = sub2(o.py, pyj);
  const float2 gix = fma2(o.s, vx, mul2(o.c, vy)), giy = fma2(o.c, nvx, mul2(o.s, vy));
  const float2 gjx = fma2(sj, vx, mul2(cj, vy)), gjy = fma2(cj, nvx, mul2(sj, vy));
  const float2 tx = fma2(gix, o.pt, a), ty = fma2(giy, o.pt, b);
  ax = fma2(mj, add2(tx, fma2(gjx, ptj, a)), ax);
  ay = fma2(mj, add2(ty, fma2(gjy, ptj, b)), ay);
  at = fma2(mj, fma2(gix, tx, mul2(giy, ty)), at);
}

// One applyJTJ pass of the block's chunk (shared by the per-step kernel and
// the persistent PCG kernel).
// The raw planes of the PCG path arrive by tensor copies (sm.bar, whose next
// phase has parity `phase`; the caller initialised it), a caller's p by
// cp.async.
template <bool MASK, bool TMA>
__device__ __forceinline__ void apply_wide_body(WideSmem& sm, const Chunk& ch, const GridProb& pr,
                                                const int* __restrict__ tiles, double* __restrict__ part,
                                                const float* __restrict__ p_in_override, int par, int update,
                                                unsigned& phase) {
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const int pl = (int)pr.plane;
  const float wfit = pr.w_fit;
  const float2 w2 = make_float2(pr.w_reg, pr.w_reg);
  const float beta = s->beta_f;
  const float2 beta2 = make_float2(beta, beta);
  const int use_beta = beta != 0.0f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const float* __restrict__ pin = p_in_override ? p_in_override : pr.p + (long long)(par & 1) * 3 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 3 * pl;
  WidePlanes pp;
  pp.src[0] = update ? pr.r : nullptr;
  pp.src[1] = update ? pr.r + pl : nullptr;
  pp.src[2] = update ? pr.r + 2 * pl : nullptr;
  pp.src[3] = update ? pr.m : nullptr;
  pp.src[4] = update ? pr.m + pl : nullptr;
  pp.src[5] = (!update || use_beta) ? pin : nullptr;
  pp.src[6] = (!update || use_beta) ? pin + pl : nullptr;
  pp.src[7] = (!update || use_beta) ? pin + 2 * pl : nullptr;
  pp.src[8] = pr.csn;
  pp.src[9] = pr.csn + pl;
  pp.src[10] = pr.c;
  pp.src[11] = pr.c + pl;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc = f2x2_zero();
  // the tile index one tile ahead and the handle range of the current tile
  // are loaded an iteration early: the inline-assembly copies order all
  // memory accesses, so a late load would stall the warp at its use
  constexpr bool tma = TMA;   // the caller checked wide_tma()
  // raw planes r0 r1 r2 m0 m1 p0 p1 p2 cos sin ux uy, all in the slab
  auto plane = [&](int k, int& z, int& m) {
    m = 0;
    z = k < 3 ? zslab(pr, 0) + k
              : k < 5 ? zslab(pr, 1) + k - 3
                      : k < 8 ? (use_beta ? zslab(pr, 2) + (par & 1) * 3 + k - 5 : -1)
                              : k < 10 ? zslab(pr, 3) + k - 8 : zslab(pr, 4) + k - 10;
  };
  auto issue = [&](int tcx) {
    if (tma) {
      if (tid == 0) tile_tma<NRAW>(sm.raw, &sm.mk, plane, MASK, pr, tile_x0(tcx, W4), tile_y0(tcx), &sm.bar);
    } else {
      wide_issue<MASK>(sm, pp, pr, tile_x0(tcx, W4), tile_y0(tcx), tid);
    }
  };
  int tc = tiles[ch.begin];
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  int hb0 = pr.hbeg[tile_id(pr, tc)], hb1 = pr.hbeg[tile_id(pr, tc) + 1];
  issue(tc);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, W4), y0 = tile_y0(tc);
    const int gx = x0 + 4 * lane, gy = y0 + ty;
    const int hcur0 = hb0, hcur1 = hb1;
    const unsigned pb = phase;
    bool ok = true;
    if (tma) {
      ok = mbar_wait(&sm.bar, pb);
      phase ^= 1u;
    } else {
      cp_async_wait_all();
    }
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar, pb);
      return;
    }
    // phase 2: staged direction, geometry and validity
    wide_stage_quad<MASK>(sm, ty + 1, lane, pr, gx, gy, update, use_beta, beta2);
    if (tid < 64) {
      const int row = tid < 32 ? 0 : HH - 1;
      wide_stage_quad<MASK>(sm, row, lane, pr, gx, y0 - 1 + row, update, use_beta, beta2);
    } else if (tid < 64 + 2 * TH) {
      const int h = tid - 64;
      const int row = 1 + (h % TH), side = h / TH;
      const int col = side ? 4 + W4 : 3;
      float a, b, c;
      if (update) {
        a = __fmul_rn(sm.raw[3].v[row][col], sm.raw[0].v[row][col]);
        b = __fmul_rn(sm.raw[3].v[row][col], sm.raw[1].v[row][col]);
        c = __fmul_rn(sm.raw[4].v[row][col], sm.raw[2].v[row][col]);
        if (use_beta) {
          a = __fmaf_rn(beta, sm.raw[5].v[row][col], a);
          b = __fmaf_rn(beta, sm.raw[6].v[row][col], b);
          c = __fmaf_rn(beta, sm.raw[7].v[row][col], c);
        }
      } else {
        a = sm.raw[5].v[row][col]; b = sm.raw[6].v[row][col]; c = sm.raw[7].v[row][col];
      }
      sm.stg[0][row][col] = a; sm.stg[1][row][col] = b; sm.stg[2][row][col] = c;
#pragma unroll
      for (int k = 0; k < 4; ++k) sm.stg[3 + k][row][col] = sm.raw[8 + k].v[row][col];
      const int hy = y0 + row - 1, hx = side ? x0 + W4 : x0 - 1;
      const bool ok = hy < pr.H && hx >= 0 && hx < pr.W;
      sm.stg[7][row][col] = (ok && (!MASK || halo_mask(sm.mk.v, row, side) == 0)) ? 1.f : 0.f;
    }
    __syncthreads();
    // the raw buffer is free: start the next tile's copies
    if (t + 1 < ch.end) {
      tc = tn;
      issue(tc);
      const int tidn = tile_id(pr, tc);
      hb0 = pr.hbeg[tidn];
      hb1 = pr.hbeg[tidn + 1];
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H) {                          // warp-uniform: one warp per row
      const long long i = (long long)gy * pr.P + gx;
      // phase 3: the stencil on two packs, A = pixels {0, 2}, B = pixels {1, 3}
      const int c = 4 + 4 * lane;
      float4 O[NSTG];
#pragma unroll
      for (int k = 0; k < NSTG; ++k) O[k] = lds4(&sm.stg[k][ty + 1][c]);
      if (update) {
        *reinterpret_cast<float4*>(pout + i) = swz4(O[0]);
        *reinterpret_cast<float4*>(pout + pl + i) = swz4(O[1]);
        *reinterpret_cast<float4*>(pout + 2 * pl + i) = swz4(O[2]);
      }
      float2 axA = make_float2(0.f, 0.f), ayA = axA, atA = axA, axB = axA, ayB = axA, atB = axA;
      const Own2 oa = {lo2(O[0]), lo2(O[1]), lo2(O[2]), lo2(O[3]), lo2(O[4]), lo2(O[5]), lo2(O[6])};
      const Own2 ob = {hi2(O[0]), hi2(O[1]), hi2(O[2]), hi2(O[3]), hi2(O[4]), hi2(O[5]), hi2(O[6])};
      {
        // horizontal neighbours: pixel -1 / 4 from the neighbouring lanes
        // (staged order: pixel 3 is .w, pixel 0 is .x) or the halo columns
        float L[NSTG], R[NSTG];
#pragma unroll
        for (int k = 0; k < NSTG; ++k) {
          L[k] = __shfl_up_sync(0xffffffffu, O[k].w, 1);
          R[k] = __shfl_down_sync(0xffffffffu, O[k].x, 1);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < NSTG; ++k) L[k] = sm.stg[k][ty + 1][3];
        }
        if (lane == 31) {
#pragma unroll
          for (int k = 0; k < NSTG; ++k) R[k] = sm.stg[k][ty + 1][4 + W4];
        }
        // A: left neighbours {-1, 1}, right neighbours {1, 3} = B
        pair2(oa, make_float2(L[0], O[0].z), make_float2(L[1], O[1].z), make_float2(L[2], O[2].z),
              make_float2(L[3], O[3].z), make_float2(L[4], O[4].z), make_float2(L[5], O[5].z),
              make_float2(L[6], O[6].z), make_float2(L[7], O[7].z), axA, ayA, atA);
        pair2(oa, ob.px, ob.py, ob.pt, ob.c, ob.s, ob.ux, ob.uy, hi2(O[7]), axA, ayA, atA);
        // B: left neighbours {0, 2} = A, right neighbours {2, 4}
        pair2(ob, oa.px, oa.py, oa.pt, oa.c, oa.s, oa.ux, oa.uy, lo2(O[7]), axB, ayB, atB);
        pair2(ob, make_float2(O[0].y, R[0]), make_float2(O[1].y, R[1]), make_float2(O[2].y, R[2]),
              make_float2(O[3].y, R[3]), make_float2(O[4].y, R[4]), make_float2(O[5].y, R[5]),
              make_float2(O[6].y, R[6]), make_float2(O[7].y, R[7]), axB, ayB, atB);
      }
#pragma unroll 1
      for (int dr = 0; dr < 2; ++dr) {        // rows above and below
        float4 U[NSTG];
        const int row = dr ? ty + 2 : ty;
#pragma unroll
        for (int k = 0; k < NSTG; ++k) U[k] = lds4(&sm.stg[k][row][c]);
        pair2(oa, lo2(U[0]), lo2(U[1]), lo2(U[2]), lo2(U[3]), lo2(U[4]), lo2(U[5]), lo2(U[6]), lo2(U[7]), axA,
              ayA, atA);
        pair2(ob, hi2(U[0]), hi2(U[1]), hi2(U[2]), hi2(U[3]), hi2(U[4]), hi2(U[5]), hi2(U[6]), hi2(U[7]), axB,
              ayB, atB);
      }
      // scale by w and the own validity, back to plain pixel order
      const float2 wa = mul2(w2, lo2(O[7])), wb = mul2(w2, hi2(O[7]));
      axA = mul2(wa, axA); ayA = mul2(wa, ayA); atA = mul2(wa, atA);
      axB = mul2(wb, axB); ayB = mul2(wb, ayB); atB = mul2(wb, atB);
      float qx[4] = {axA.x, axB.x, axA.y, axB.y};
      float qy[4] = {ayA.x, ayB.x, ayA.y, ayB.y};
      float qt[4] = {atA.x, atB.x, atA.y, atB.y};
      const float vf[4] = {O[7].x, O[7].z, O[7].y, O[7].w};
      const float4 opx = swz4(O[0]), opy = swz4(O[1]), opt = swz4(O[2]);
      // explicit roundings (no contraction left to the compiler), so that
      // every kernel instantiating this body computes the same bits
      for (int h = hcur0; h < hcur1; ++h) {
        const long long k = pr.hpix[h] - i;
        if (k >= 0 && k < 4) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk == k && vf[kk] != 0.f) {
              qx[kk] = __fmaf_rn(wfit, cmp(opx, kk), qx[kk]);
              qy[kk] = __fmaf_rn(wfit, cmp(opy, kk), qy[kk]);
            }
        }
      }
      if (pr.lm) {
        const float4 dd = ld4(pr.dc + i), dt = ld4(pr.dc + pl + i);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (vf[k] == 0.f) continue;
          qx[k] = __fmaf_rn(__fmul_rn(lam, cmp(dd, k)), cmp(opx, k), qx[k]);
          qy[k] = __fmaf_rn(__fmul_rn(lam, cmp(dd, k)), cmp(opy, k), qy[k]);
          qt[k] = __fmaf_rn(__fmul_rn(lam, cmp(dt, k)), cmp(opt, k), qt[k]);
        }
      }
      *reinterpret_cast<float4*>(pr.q + i) = make_float4(qx[0], qx[1], qx[2], qx[3]);
      *reinterpret_cast<float4*>(pr.q + pl + i) = make_float4(qy[0], qy[1], qy[2], qy[3]);
      *reinterpret_cast<float4*>(pr.q + 2 * pl + i) = make_float4(qt[0], qt[1], qt[2], qt[3]);
      f2x2_add_prod(acc, lo2(opx), make_float2(qx[0], qx[1]));
      f2x2_add_prod(acc, hi2(opx), make_float2(qx[2], qx[3]));
      f2x2_add_prod(acc, lo2(opy), make_float2(qy[0], qy[1]));
      f2x2_add_prod(acc, hi2(opy), make_float2(qy[2], qy[3]));
      f2x2_add_prod(acc, lo2(opt), make_float2(qt[0], qt[1]));
      f2x2_add_prod(acc, hi2(opt), make_float2(qt[2], qt[3]));
    }
  }
  cp_async_wait_all();
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc), f2_zero(), &s->counter, pr.chunk_end - pr.chunk_begin)) {
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

template <bool MASK>
__global__ void __launch_bounds__(NT, 2) k_warp_apply_wide(const GridProb* __restrict__ probs,
                                                           const Chunk* __restrict__ chunks,
                                                           const int* __restrict__ tiles,
                                                           double* __restrict__ part,
                                                           const float* __restrict__ p_in_override,
                                                           int par, int update) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  WideSmem& sm = *reinterpret_cast<WideSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (threadIdx.x == 0) mbar_init(&sm.bar);
  __syncthreads();
  unsigned phase = 0;
  // the PCG path stages by tensor copies, a caller's p (the J^T J p hook) by cp.async
  if (update && !p_in_override && wide_tma(pr, &sm))
    apply_wide_body<MASK, true>(sm, ch, pr, tiles, part, p_in_override, par, update, phase);
  else
    apply_wide_body<MASK, false>(sm, ch, pr, tiles, part, p_in_override, par, update, phase);
}

// cos / sin of the new theta quad into the cos / sin planes (wide warps: the
// next PCGInit reads them instead of evaluating them on its tile and halo)
__device__ __forceinline__ void store_csn(const GridProb& pr, long long i, const float4& th) {
  float4 cs, sn;
  sincosf(th.x, &sn.x, &cs.x);
  sincosf(th.y, &sn.y, &cs.y);
  sincosf(th.z, &sn.z, &cs.z);
  sincosf(th.w, &sn.w, &cs.w);
  *reinterpret_cast<float4*>(pr.csn + i) = cs;
  *reinterpret_cast<float4*>(pr.csn + pr.plane + i) = sn;
}

// ---------------------------------------------------------------------------
// Single-reduction PCG iteration of the wide warp (tw = 128): one launch per
// PCG iteration instead of applyJTJ + vector update.  The Jacobi-PCG of
// Sec. 4.1 needs two grid-wide reductions per iteration (p.q for alpha, then
// r.z for beta), so its update and the next direction normally sit in two
// launches.  Here the kernel of iteration i forms, in one reduction, p.q,
// q.z, q.M^-1 q and r.z (r = z / M^-1, the residual the stored z stands
// for, in iteration 0 as well).  Its last block sets
//   alpha_i = rz_i / pq_i,
//   rz_{i+1} = (r_i - alpha_i q_i) . M^-1 (r_i - alpha_i q_i)
//            = rz_i - 2 alpha_i (q_i . z_i) + alpha_i^2 (q_i . M^-1 q_i),
//   beta_{i+1} = rz_{i+1} / rz_i
// (the recurrence of single-synchronisation CG variants such as Chronopoulos
// & Gear's; the same Krylov iterates as the two-pass form in exact
// arithmetic).  The recurrence only sets beta: alpha always divides the r.z
// measured on the stored vectors, so that once the residual reaches the
// float32 rounding floor (where the recurrence is dominated by rounding) the
// steps stay at rounding size.  The vector update of iteration i - 1 moves
// into the kernel of iteration i, which forms on its tile and halo
//   z_i = z_{i-1} - alpha_{i-1} w_{i-1}       (w = M^-1 q, so z = M^-1 r)
//   p_i = z_i + beta_i p_{i-1}
// and on its own pixels delta += alpha_{i-1} p_{i-1}, q_i = (J^T J + lambda D)
// p_i, w_i = M^-1 q_i.  r and q themselves are never stored.  z, w and p are
// double-buffered (halo reads of the previous iterate while other blocks
// write the next).  Iteration 0 starts from r_0 and M^-1 (z_0 = M^-1 r_0, p_0
// = z_0); the last iteration's update is applied by k_grid_fused_fin (for
// Gauss-Newton together with the outer update x += delta).
// Per pixel: read z, w, p (halos), cos / sin, UrShape, M^-1, delta; write z,
// w, p, delta: 120 B against 152 B for the two-pass form.
// Breakdown (p.q <= 0 or r.z = 0, or a recurrence r.z <= 0) stops the loop
// as in the two-pass form; a step whose alpha is known is still applied.
// ---------------------------------------------------------------------------
constexpr int NRAW_F = 13;       // z0 z1 z2 w0 w1 w2 p0 p1 p2 cos sin ux uy (iteration 0: r0 r1 r2 m0 m1 at 0..4)
constexpr int NSTG_F = 7;        // px py pt cos sin ux uy, each quad stored as pixels 0 2 1 3

struct FusedSmem {
  PlaneT raw[NRAW_F];
  float stg[NSTG_F][HH][SP];     // halo columns -1 / 128 live at 3 / 132, in plain order
  BytesT mk[2];                  // masked problems: byte plane of the current / next tile
  unsigned long long bar;
};

// a x + y and a * b per lane, as packed float32 pairs (correctly rounded per
// lane: the same bits as scalar fmaf / fmul)
__device__ __forceinline__ float4 fma4s(float a, const float4& x, const float4& y) {
  return fma4p(make_float2(a, a), x, y);
}
__device__ __forceinline__ float4 mul4s(const float4& a, const float4& b) { return mul4p(a, b); }
__device__ __forceinline__ float2 valid2(bool a, bool b) { return make_float2(a ? 1.f : 0.f, b ? 1.f : 0.f); }
// approximate reciprocal (the PTX rcp.approx instruction: one special-function
// op, a few ulp): r = z / M^-1 only feeds the r.z that alpha divides, which is
// rounded to float32 anyway
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float4 rcp4(const float4& v) {
  return make_float4(rcp_approx(v.x), rcp_approx(v.y), rcp_approx(v.z), rcp_approx(v.w));
}

// Pending-only pass: the loop stopped after an iteration whose step is known
// (alpha != 0): delta += alpha p over the block's pixels, and the last block
// clears alpha.
template <int NX>
__device__ __forceinline__ void fused_pending(const Chunk& ch, const GridProb& pr, const int* __restrict__ tiles,
                                              double* __restrict__ part, const float* __restrict__ pin,
                                              float alpha) {
  Scalars* s = pr.s;
  const long long pl = pr.plane;
  constexpr int QPT = (W4 / 4) * TH;
  const int nq = (ch.end - ch.begin) * QPT;
  for (int k = threadIdx.x; k < nq; k += NT) {
    const int tc = tiles[ch.begin + k / QPT];
    const int w = k % QPT;
    const int y = tile_y0(tc) + w / (W4 / 4);
    if (y >= pr.H) continue;
    const long long i = (long long)y * pr.P + tile_x0(tc, W4) + 4 * (w % (W4 / 4));
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      float4* d = reinterpret_cast<float4*>(pr.d + c * pl + i);
      *d = fma4s(alpha, __ldcg(reinterpret_cast<const float4*>(pin + c * pl + i)), *d);
    }
  }
  const F2 none[4] = {f2_zero(), f2_zero(), f2_zero(), f2_zero()};
  if (publish_partials4(part, blockIdx.x, none, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double unused[4];
    gather_partials4(part, pr.chunk_begin, pr.chunk_end, &s->counter, unused);
    if (threadIdx.x == 0) s->alpha_f = 0.f;
  }
}

// End of a single-reduction iteration: the block's four compensated sums
// (p.q, q.z, q.M^-1 q, r.z) published; the last block of the problem sets
// alpha, the next r.z and beta (or ends the loop on a breakdown).
__device__ __forceinline__ void fused_finish(const GridProb& pr, double* __restrict__ part, const F2x2& acc_pq,
                                             const F2x2& acc_qz, const F2x2& acc_qw, const F2x2& acc_zr) {
  Scalars* s = pr.s;
  const F2 sums[4] = {f2x2_fold(acc_pq), f2x2_fold(acc_qz), f2x2_fold(acc_qw), f2x2_fold(acc_zr)};
  if (publish_partials4(part, blockIdx.x, sums, &s->counter, pr.chunk_end - pr.chunk_begin)) {
    double v[4];
    gather_partials4(part, pr.chunk_begin, pr.chunk_end, &s->counter, v);
    if (threadIdx.x == 0) {
      const double pq = v[0], qz = v[1], qw = v[2], rz = v[3];
      s->pq = pq;
      if (pq > 0.0 && isfinite(pq) && rz > 0.0 && isfinite(rz)) {
        // alpha from the r.z of the stored z (as the two-pass form takes it);
        // the recurrence only carries r.z one iteration ahead, to set beta
        const float af = (float)(rz / pq);
        const double a = (double)af;
        const double rz_next = fma(a * a, qw, fma(-2.0 * a, qz, rz));
        s->alpha_f = af;
        s->rz = rz;
        s->pcg_iters += 1;
        if (rz_next > 0.0 && isfinite(rz_next)) {
          s->beta_f = (float)(rz_next / rz);
        } else {
          s->pcg_active = 0;        // the step alpha p is still applied
          if (!isfinite(rz_next)) s->nonfinite = 1;
        }
      } else {
        s->alpha_f = 0.f;
        s->pcg_active = 0;
        if (!isfinite(pq) || !isfinite(rz)) s->nonfinite = 1;
      }
    }
  }
}

// One single-reduction PCG iteration `it` of the block's chunk (staged by
// tensor copies, like the wide apply).
template <bool MASK>
__device__ __forceinline__ void fused_wide_body(FusedSmem& sm, const Chunk& ch, const GridProb& pr,
                                                const int* __restrict__ tiles, double* __restrict__ part, int it) {
  Scalars* s = pr.s;
  if (s->done) return;
  const int first = it == 0;
  const float alpha = first ? 0.f : s->alpha_f;
  const long long pl = pr.plane;
  const float* __restrict__ pin = pr.p + (long long)(it & 1) * 3 * pl;
  if (!s->pcg_active) {
    if (alpha != 0.f) fused_pending<3>(ch, pr, tiles, part, pin, alpha);
    return;
  }
  const float beta = first ? 0.f : s->beta_f;
  const int use_beta = beta != 0.0f;
  const float wfit = pr.w_fit;
  const float2 w2 = make_float2(pr.w_reg, pr.w_reg);
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  float* __restrict__ pout = pr.p + (long long)((it + 1) & 1) * 3 * pl;
  float* __restrict__ zout = pr.zb + (long long)((it + 1) & 1) * 3 * pl;
  float* __restrict__ wout = pr.wb + (long long)((it + 1) & 1) * 3 * pl;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc_pq = f2x2_zero(), acc_qz = f2x2_zero(), acc_qw = f2x2_zero(), acc_zr = f2x2_zero();
  const int zz = pr.zpack2 & 63, zw = (pr.zpack2 >> 6) & 63, par3 = (it & 1) * 3;
  // raw planes, all in the slab (tensor map 0)
  auto plane = [&](int k, int& z, int& m) {
    m = 0;
    if (k >= 9) {
      z = k < 11 ? zslab(pr, 3) + k - 9 : zslab(pr, 4) + k - 11;
    } else if (first) {
      z = k < 3 ? zslab(pr, 0) + k : k < 5 ? zslab(pr, 1) + k - 3 : -1;
    } else {
      z = k < 3 ? zz + par3 + k : k < 6 ? zw + par3 + k - 3 : zslab(pr, 2) + par3 + k - 6;
    }
  };
  auto issue = [&](int tcx, int slot) {
    if (tid == 0) tile_tma<NRAW_F>(sm.raw, &sm.mk[slot], plane, MASK, pr, tile_x0(tcx, W4), tile_y0(tcx), &sm.bar);
  };
  // direction and z of one quad of staged row `row` (column c); ownrow:
  // also the z / delta stores of the thread's own pixels
  // delta of the thread's own pixels, loaded before the staging wait
  float4 dl[3];
  auto stage = [&](int row, int gy, bool own, long long i) {
    const int c = 4 + 4 * lane;
    auto R = [&](int k) { return lds4(&sm.raw[k].v[row][c]); };
    float4 zx, zy, zt;
    if (first) {
      const float4 m0 = R(3), m1 = R(4);
      zx = mul4s(m0, R(0)); zy = mul4s(m0, R(1)); zt = mul4s(m1, R(2));
    } else {
      zx = fma4s(-alpha, R(3), R(0)); zy = fma4s(-alpha, R(4), R(1)); zt = fma4s(-alpha, R(5), R(2));
    }
    float4 px = zx, py = zy, pt = zt;
    if (use_beta) {
      px = fma4s(beta, R(6), zx); py = fma4s(beta, R(7), zy); pt = fma4s(beta, R(8), zt);
    }
    sts4(&sm.stg[0][row][c], swz4(px));
    sts4(&sm.stg[1][row][c], swz4(py));
    sts4(&sm.stg[2][row][c], swz4(pt));
#pragma unroll
    for (int k = 0; k < 4; ++k) sts4(&sm.stg[3 + k][row][c], swz4(R(9 + k)));
    if (own && gy < pr.H) {
      *reinterpret_cast<float4*>(zout + i) = zx;
      *reinterpret_cast<float4*>(zout + pl + i) = zy;
      *reinterpret_cast<float4*>(zout + 2 * pl + i) = zt;
      if (!first) {
        *reinterpret_cast<float4*>(pr.d + i) = fma4s(alpha, R(6), dl[0]);
        *reinterpret_cast<float4*>(pr.d + pl + i) = fma4s(alpha, R(7), dl[1]);
        *reinterpret_cast<float4*>(pr.d + 2 * pl + i) = fma4s(alpha, R(8), dl[2]);
      }
    }
  };
  int tc = tiles[ch.begin];
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  int hb0 = pr.hbeg[tile_id(pr, tc)], hb1 = pr.hbeg[tile_id(pr, tc) + 1];
  unsigned phase = 0;
  int slot = 0;
  issue(tc, 0);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, W4), y0 = tile_y0(tc);
    const int gx = x0 + 4 * lane, gy = y0 + ty;
    const long long i = (long long)gy * pr.P + gx;
    const int hcur0 = hb0, hcur1 = hb1;
    if (!first && gy < pr.H) {
#pragma unroll
      for (int k = 0; k < 3; ++k) dl[k] = *reinterpret_cast<const float4*>(pr.d + k * pl + i);
    }
    const unsigned pb = phase;
    const bool ok = mbar_wait(&sm.bar, pb);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar, pb);
      return;
    }
    const unsigned char (*mk)[SPB] = sm.mk[slot].v;
    // phase 2: z and the direction on the tile and its halo
    stage(ty + 1, gy, true, i);
    if (tid < 64) {
      const int row = tid < 32 ? 0 : HH - 1;
      stage(row, y0 - 1 + row, false, 0);
    } else if (tid < 64 + 2 * TH) {
      const int h = tid - 64;
      const int row = 1 + (h % TH), side = h / TH;
      const int col = side ? 4 + W4 : 3;
      auto R = [&](int k) { return sm.raw[k].v[row][col]; };
      float zx, zy, zt;
      if (first) {
        zx = __fmul_rn(R(3), R(0)); zy = __fmul_rn(R(3), R(1)); zt = __fmul_rn(R(4), R(2));
      } else {
        zx = __fmaf_rn(-alpha, R(3), R(0)); zy = __fmaf_rn(-alpha, R(4), R(1)); zt = __fmaf_rn(-alpha, R(5), R(2));
      }
      if (use_beta) {
        zx = __fmaf_rn(beta, R(6), zx); zy = __fmaf_rn(beta, R(7), zy); zt = __fmaf_rn(beta, R(8), zt);
      }
      sm.stg[0][row][col] = zx; sm.stg[1][row][col] = zy; sm.stg[2][row][col] = zt;
#pragma unroll
      for (int k = 0; k < 4; ++k) sm.stg[3 + k][row][col] = R(9 + k);
    }
    __syncthreads();
    // the raw buffer is free: start the next tile's copies
    if (t + 1 < ch.end) {
      tc = tn;
      issue(tc, slot ^ 1);
      const int tidn = tile_id(pr, tc);
      hb0 = pr.hbeg[tidn];
      hb1 = pr.hbeg[tidn + 1];
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H) {                          // warp-uniform: one warp per row
      const int c = 4 + 4 * lane;
      float4 O[NSTG_F];
#pragma unroll
      for (int k = 0; k < NSTG_F; ++k) O[k] = lds4(&sm.stg[k][ty + 1][c]);
      *reinterpret_cast<float4*>(pout + i) = swz4(O[0]);
      *reinterpret_cast<float4*>(pout + pl + i) = swz4(O[1]);
      *reinterpret_cast<float4*>(pout + 2 * pl + i) = swz4(O[2]);
      // validity of the own pixels and of their neighbours (1 / 0): inside
      // the grid and, with a mask, not excluded; staged order 0 2 1 3
      float2 vA, vB, lA, rA, rB, up2A, up2B, dn2A, dn2B;
      {
        const bool upok = gy > 0, dnok = gy + 1 < pr.H;
        if (!MASK) {
          vA = valid2(gx < pr.W, gx + 2 < pr.W);
          vB = valid2(gx + 1 < pr.W, gx + 3 < pr.W);
          lA = valid2(gx > 0, true);
          rA = vB;
          rB = valid2(gx + 2 < pr.W, gx + 4 < pr.W);
          up2A = up2B = valid2(upok, upok);
          dn2A = dn2B = valid2(dnok, dnok);
        } else {
          // byte of column x0 + k at mk[row][16 + k]; halo columns at 15 / 144
          auto fr = [&](int row, int k) {
            return gx + k >= 0 && gx + k < pr.W && mk[row][16 + 4 * lane + k] == 0;
          };
          const int ro = ty + 1;
          vA = valid2(fr(ro, 0), fr(ro, 2));
          vB = valid2(fr(ro, 1), fr(ro, 3));
          lA = valid2(gx > 0 && mk[ro][15 + 4 * lane] == 0, fr(ro, 1));
          rA = vB;
          rB = valid2(fr(ro, 2), gx + 4 < pr.W && mk[ro][20 + 4 * lane] == 0);
          up2A = valid2(upok && fr(ro - 1, 0), upok && fr(ro - 1, 2));
          up2B = valid2(upok && fr(ro - 1, 1), upok && fr(ro - 1, 3));
          dn2A = valid2(dnok && fr(ro + 1, 0), dnok && fr(ro + 1, 2));
          dn2B = valid2(dnok && fr(ro + 1, 1), dnok && fr(ro + 1, 3));
        }
      }
      float2 axA = make_float2(0.f, 0.f), ayA = axA, atA = axA, axB = axA, ayB = axA, atB = axA;
      const Own2 oa = {lo2(O[0]), lo2(O[1]), lo2(O[2]), lo2(O[3]), lo2(O[4]), lo2(O[5]), lo2(O[6])};
      const Own2 ob = {hi2(O[0]), hi2(O[1]), hi2(O[2]), hi2(O[3]), hi2(O[4]), hi2(O[5]), hi2(O[6])};
      {
        float L[NSTG_F], R[NSTG_F];
#pragma unroll
        for (int k = 0; k < NSTG_F; ++k) {
          L[k] = __shfl_up_sync(0xffffffffu, O[k].w, 1);
          R[k] = __shfl_down_sync(0xffffffffu, O[k].x, 1);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < NSTG_F; ++k) L[k] = sm.stg[k][ty + 1][3];
        }
        if (lane == 31) {
#pragma unroll
          for (int k = 0; k < NSTG_F; ++k) R[k] = sm.stg[k][ty + 1][4 + W4];
        }
        pair2(oa, make_float2(L[0], O[0].z), make_float2(L[1], O[1].z), make_float2(L[2], O[2].z),
              make_float2(L[3], O[3].z), make_float2(L[4], O[4].z), make_float2(L[5], O[5].z),
              make_float2(L[6], O[6].z), lA, axA, ayA, atA);
        pair2(oa, ob.px, ob.py, ob.pt, ob.c, ob.s, ob.ux, ob.uy, rA, axA, ayA, atA);
        pair2(ob, oa.px, oa.py, oa.pt, oa.c, oa.s, oa.ux, oa.uy, vA, axB, ayB, atB);
        pair2(ob, make_float2(O[0].y, R[0]), make_float2(O[1].y, R[1]), make_float2(O[2].y, R[2]),
              make_float2(O[3].y, R[3]), make_float2(O[4].y, R[4]), make_float2(O[5].y, R[5]),
              make_float2(O[6].y, R[6]), rB, axB, ayB, atB);
      }
#pragma unroll 1
      for (int dr = 0; dr < 2; ++dr) {        // rows above and below
        float4 U[NSTG_F];
        const int row = dr ? ty + 2 : ty;
#pragma unroll
        for (int k = 0; k < NSTG_F; ++k) U[k] = lds4(&sm.stg[k][row][c]);
        const float2 mA = dr ? dn2A : up2A, mB = dr ? dn2B : up2B;
        pair2(oa, lo2(U[0]), lo2(U[1]), lo2(U[2]), lo2(U[3]), lo2(U[4]), lo2(U[5]), lo2(U[6]), mA, axA, ayA, atA);
        pair2(ob, hi2(U[0]), hi2(U[1]), hi2(U[2]), hi2(U[3]), hi2(U[4]), hi2(U[5]), hi2(U[6]), mB, axB, ayB, atB);
      }
      const float2 wa = mul2(w2, vA), wb = mul2(w2, vB);
      axA = mul2(wa, axA); ayA = mul2(wa, ayA); atA = mul2(wa, atA);
      axB = mul2(wb, axB); ayB = mul2(wb, ayB); atB = mul2(wb, atB);
      float qx[4] = {axA.x, axB.x, axA.y, axB.y};
      float qy[4] = {ayA.x, ayB.x, ayA.y, ayB.y};
      float qt[4] = {atA.x, atB.x, atA.y, atB.y};
      const float vf[4] = {vA.x, vB.x, vA.y, vB.y};
      const float4 opx = swz4(O[0]), opy = swz4(O[1]), opt = swz4(O[2]);
      for (int h = hcur0; h < hcur1; ++h) {
        const long long k = pr.hpix[h] - i;
        if (k >= 0 && k < 4) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk == k && vf[kk] != 0.f) {
              qx[kk] = __fmaf_rn(wfit, cmp(opx, kk), qx[kk]);
              qy[kk] = __fmaf_rn(wfit, cmp(opy, kk), qy[kk]);
            }
        }
      }
      if (pr.lm) {
        const float4 dd = ld4(pr.dc + i), dt = ld4(pr.dc + pl + i);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (vf[k] == 0.f) continue;
          qx[k] = __fmaf_rn(__fmul_rn(lam, cmp(dd, k)), cmp(opx, k), qx[k]);
          qy[k] = __fmaf_rn(__fmul_rn(lam, cmp(dd, k)), cmp(opy, k), qy[k]);
          qt[k] = __fmaf_rn(__fmul_rn(lam, cmp(dt, k)), cmp(opt, k), qt[k]);
        }
      }
      // w = M^-1 q and the three inner products; z of the own pixels comes
      // back from the stores of phase 2 (this thread's own writes)
      const float4 m0 = ld4(pr.m + i), m1 = ld4(pr.m + pl + i);
      const float4 qxv = make_float4(qx[0], qx[1], qx[2], qx[3]);
      const float4 qyv = make_float4(qy[0], qy[1], qy[2], qy[3]);
      const float4 qtv = make_float4(qt[0], qt[1], qt[2], qt[3]);
      const float4 wx = mul4s(m0, qxv), wy = mul4s(m0, qyv), wt = mul4s(m1, qtv);
      *reinterpret_cast<float4*>(wout + i) = wx;
      *reinterpret_cast<float4*>(wout + pl + i) = wy;
      *reinterpret_cast<float4*>(wout + 2 * pl + i) = wt;
      const float4 zxv = *reinterpret_cast<const float4*>(zout + i);
      const float4 zyv = *reinterpret_cast<const float4*>(zout + pl + i);
      const float4 ztv = *reinterpret_cast<const float4*>(zout + 2 * pl + i);
      f2x2_add_prod(acc_pq, lo2(opx), lo2(qxv)); f2x2_add_prod(acc_pq, hi2(opx), hi2(qxv));
      f2x2_add_prod(acc_pq, lo2(opy), lo2(qyv)); f2x2_add_prod(acc_pq, hi2(opy), hi2(qyv));
      f2x2_add_prod(acc_pq, lo2(opt), lo2(qtv)); f2x2_add_prod(acc_pq, hi2(opt), hi2(qtv));
      f2x2_add_prod(acc_qw, lo2(wx), lo2(qxv)); f2x2_add_prod(acc_qw, hi2(wx), hi2(qxv));
      f2x2_add_prod(acc_qw, lo2(wy), lo2(qyv)); f2x2_add_prod(acc_qw, hi2(wy), hi2(qyv));
      f2x2_add_prod(acc_qw, lo2(wt), lo2(qtv)); f2x2_add_prod(acc_qw, hi2(wt), hi2(qtv));
      f2x2_add_prod(acc_qz, lo2(zxv), lo2(qxv)); f2x2_add_prod(acc_qz, hi2(zxv), hi2(qxv));
      f2x2_add_prod(acc_qz, lo2(zyv), lo2(qyv)); f2x2_add_prod(acc_qz, hi2(zyv), hi2(qyv));
      f2x2_add_prod(acc_qz, lo2(ztv), lo2(qtv)); f2x2_add_prod(acc_qz, hi2(ztv), hi2(qtv));
      // r.z of the own pixels, with r = z / M^-1
      const float4 d0 = rcp4(m0), d1 = rcp4(m1);
      const float4 rx = mul4s(d0, zxv), ry = mul4s(d0, zyv), rt = mul4s(d1, ztv);
      f2x2_add_prod(acc_zr, lo2(zxv), lo2(rx)); f2x2_add_prod(acc_zr, hi2(zxv), hi2(rx));
      f2x2_add_prod(acc_zr, lo2(zyv), lo2(ry)); f2x2_add_prod(acc_zr, hi2(zyv), hi2(ry));
      f2x2_add_prod(acc_zr, lo2(ztv), lo2(rt)); f2x2_add_prod(acc_zr, hi2(ztv), hi2(rt));
    }
    slot ^= 1;
  }
  fused_finish(pr, part, acc_pq, acc_qz, acc_qw, acc_zr);
}

template <bool MASK>
__global__ void __launch_bounds__(NT, 2) k_warp_fused_wide(const GridProb* __restrict__ probs,
                                                           const Chunk* __restrict__ chunks,
                                                           const int* __restrict__ tiles,
                                                           double* __restrict__ part, int it) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  FusedSmem& sm = *reinterpret_cast<FusedSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (threadIdx.x == 0) mbar_init(&sm.bar);
  __syncthreads();
  if (tma_ready(pr, &sm)) fused_wide_body<MASK>(sm, ch, pr, tiles, part, it);
}

// After the last single-reduction iteration: delta += alpha p for the step
// whose alpha is known (p of parity `par`), unless the loop has none pending.
// step = 1 (Gauss-Newton): the outer update x += delta follows in the same
// pass (the same roundings as the update, then k_grid_step), and delta is
// not stored; csn_out: also cos / sin of the new theta.
template <int NX>
__global__ void __launch_bounds__(NT) k_grid_fused_fin(const GridProb* __restrict__ probs,
                                                       const Chunk* __restrict__ chunks,
                                                       const int* __restrict__ tiles, int par, int step,
                                                       int csn_out) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  const Scalars* s = pr.s;
  if (s->done) return;
  const float alpha = s->alpha_f;
  if (alpha == 0.f && !step) return;
  const long long pl = pr.plane;
  const float* __restrict__ pin = pr.p + (long long)(par & 1) * NX * pl;
  constexpr int QPT = (W4 / 4) * TH;
  const int nq = (ch.end - ch.begin) * QPT;
  for (int k = threadIdx.x; k < nq; k += NT) {
    const int tc = tiles[ch.begin + k / QPT];
    const int w = k % QPT;
    const int y = tile_y0(tc) + w / (W4 / 4);
    if (y >= pr.H) continue;
    const long long i = (long long)y * pr.P + tile_x0(tc, W4) + 4 * (w % (W4 / 4));
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      float4* d = reinterpret_cast<float4*>(pr.d + c * pl + i);
      float4 dv = *d;
      if (alpha != 0.f) dv = fma4s(alpha, __ldcg(reinterpret_cast<const float4*>(pin + c * pl + i)), dv);
      if (step) {
        float4* x = reinterpret_cast<float4*>(pr.x + c * pl + i);
        float4 xv = *x;
        xv = make_float4(xv.x + dv.x, xv.y + dv.y, xv.z + dv.z, xv.w + dv.w);
        *x = xv;
        if (NX == 3 && c == 2 && csn_out) store_csn(pr, i, xv);
      } else {
        *d = dv;
      }
    }
  }
}

// Wide-tile warp PCGInit (tw = 128), staged like the wide apply: tensor
// copies bring the raw planes (dx, dy, theta, UrShape) of the halo-extended
// tile into shared memory, phase 2 evaluates cos / sin of theta once per
// staged pixel, then the next tile's copies overlap phase 3.  Per valid neighbour
// pair (i, j), with a = d_i - d_j, v = U_i - U_j, e_k = v - R(theta_k) v and
// G_i = -R'(theta_i) v:
//   own residual       r_(i,j) =  s_w (a + e_i)
//   incoming residual  r_(j,i) = -s_w (a + e_j)
//   J^T F (d rows)  += w (2 a + e_i + e_j),   J^T F (theta row) += w G_i . (a + e_i)
//   diag (d rows)   += 2 w,                   diag (theta row)  += w |G_i|^2
//   E               += w |a + e_i|^2   (own residuals only)
// Writes r = b = -J^T F, M^-1, delta = 0, the LM diagonal, cos / sin of theta.
constexpr int NRAW_I = 6;        // dx dy theta ux uy (-), or with cos / sin read: dx dy cos ux uy sin
constexpr int NSTG_I = 7;        // dx dy cos sin ux uy valid, quads stored as pixels 0 2 1 3

struct InitSmem {
  PlaneT raw[NRAW_I];
  float stg[NSTG_I][HH][SP];     // halo columns -1 / 128 live at 3 / 132, in plain order
  BytesT mk;
  unsigned long long bar;        // tensor-copy completion of the raw planes
};

// Phase 2 for one staged quad: cos / sin of theta (evaluated, or with CSN
// copied from the planes the previous outer update wrote), copied values,
// validity, in the staged order 0 2 1 3.
template <bool MASK, bool CSN>
__device__ __forceinline__ void init_stage_quad(InitSmem& sm, int row, int lane, const GridProb& pr, int gx, int gy) {
  const int c = 4 + 4 * lane;
  float4 cs, sn;
  if (CSN) {
    cs = lds4(&sm.raw[2].v[row][c]);
    sn = lds4(&sm.raw[5].v[row][c]);
  } else {
    const float4 th = lds4(&sm.raw[2].v[row][c]);
    sincosf(th.x, &sn.x, &cs.x);
    sincosf(th.y, &sn.y, &cs.y);
    sincosf(th.z, &sn.z, &cs.z);
    sincosf(th.w, &sn.w, &cs.w);
  }
  sts4(&sm.stg[0][row][c], swz4(lds4(&sm.raw[0].v[row][c])));
  sts4(&sm.stg[1][row][c], swz4(lds4(&sm.raw[1].v[row][c])));
  sts4(&sm.stg[2][row][c], swz4(cs));
  sts4(&sm.stg[3][row][c], swz4(sn));
  sts4(&sm.stg[4][row][c], swz4(lds4(&sm.raw[3].v[row][c])));
  sts4(&sm.stg[5][row][c], swz4(lds4(&sm.raw[4].v[row][c])));
  float vk[4] = {0.f, 0.f, 0.f, 0.f};
  if (gy >= 0 && gy < pr.H) {
    const unsigned int m4 = MASK ? *reinterpret_cast<const unsigned int*>(&sm.mk.v[row][16 + 4 * lane]) : 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      vk[k] = (gx + k < pr.W && (!MASK || ((m4 >> (8 * k)) & 0xffu) == 0u)) ? 1.f : 0.f;
  }
  sts4(&sm.stg[6][row][c], make_float4(vk[0], vk[2], vk[1], vk[3]));
}

// Own values of one float2 pack for PCGInit.
struct OwnI2 {
  float2 dx, dy, c, s, ux, uy;
};
struct AccI2 {
  float2 gx, gy, gt, dt, e, np;
};

// Grouped J^T F / diag / energy terms of the pairs (i, j) of one pack, scaled
// by the neighbour's validity m_j.  With v = U_i - U_j, a = d_i - d_j and
// G_k = (s_k v_x + c_k v_y, s_k v_y - c_k v_x), the rotation residual part is
// e_k = v - R(theta_k) v = (v_x + G_k,y, v_y - G_k,x), own residual / s_w
// o = a + e_i:
//   J^T F_d += o + (a + e_j),  J^T F_t += G_i . o,  diag_t += |G_i|^2,
//   E += |o|^2,  np += 1 (diag_d = 2 w np).
__device__ __forceinline__ void init_pair2(const OwnI2& o, float2 dxj, float2 dyj, float2 cj, float2 sj, float2 uxj,
                                           float2 uyj, float2 mj, AccI2& A) {
  const float2 vx = sub2(o.ux, uxj), vy = sub2(o.uy, uyj), nvx = sub2(uxj, o.ux);
  const float2 ax = sub2(o.dx, dxj), ay = sub2(o.dy, dyj);
  const float2 gix = fma2(o.s, vx, mul2(o.c, vy)), giy = fma2(o.s, vy, mul2(o.c, nvx));
  const float2 gjx = fma2(sj, vx, mul2(cj, vy)), gjy = fma2(sj, vy, mul2(cj, nvx));
  const float2 ox = add2(ax, add2(vx, giy)), oy = add2(ay, sub2(vy, gix));
  const float2 fx = add2(ox, add2(ax, add2(vx, gjy))), fy = add2(oy, add2(ay, sub2(vy, gjx)));
  A.gx = fma2(mj, fx, A.gx);
  A.gy = fma2(mj, fy, A.gy);
  A.gt = fma2(mj, fma2(gix, ox, mul2(giy, oy)), A.gt);
  A.dt = fma2(mj, fma2(gix, gix, mul2(giy, giy)), A.dt);
  A.e = fma2(mj, fma2(ox, ox, mul2(oy, oy)), A.e);
  A.np = add2(A.np, mj);
}

template <bool MASK, bool CSN>
__device__ __forceinline__ void k_warp_init_wide_body(InitSmem& sm, const Chunk& ch, const GridProb& pr,
    const int* __restrict__ tiles, double* __restrict__ part, int k_outer, float dmin, float dmax) {
  Scalars* s = pr.s;
  if (s->done) return;
  const int pl = (int)pr.plane;
  const float w = pr.w_reg, wfit = pr.w_fit;
  const float2 w2 = make_float2(w, w);
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc_rz = f2x2_zero(), acc_E = f2x2_zero();
  // raw planes by tensor copies: dx, dy, theta from the unknowns, UrShape
  // from the slab; with CSN cos / sin (slab) in place of theta
  auto plane = [&](int k, int& z, int& m) {
    m = (k < 2 || (k == 2 && !CSN)) ? 1 : 0;
    z = k < 2 ? k : k == 2 ? (CSN ? zslab(pr, 3) : 2) : k < 5 ? zslab(pr, 4) + k - 3 : (CSN ? zslab(pr, 3) + 1 : -1);
  };
  if (tid == 0) mbar_init(&sm.bar);
  __syncthreads();
  auto issue = [&](int tcx) {
    if (tid == 0) tile_tma<NRAW_I>(sm.raw, &sm.mk, plane, MASK, pr, tile_x0(tcx, W4), tile_y0(tcx), &sm.bar);
  };
  unsigned phase = 0;
  int tc = tiles[ch.begin];
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  int hb0 = pr.hbeg[tile_id(pr, tc)], hb1 = pr.hbeg[tile_id(pr, tc) + 1];
  issue(tc);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, W4), y0 = tile_y0(tc);
    const int gx = x0 + 4 * lane, gy = y0 + ty;
    const int hcur0 = hb0, hcur1 = hb1;
    const unsigned pb = phase;
    const bool ok = mbar_wait(&sm.bar, pb);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar, pb);
      return;
    }
    init_stage_quad<MASK, CSN>(sm, ty + 1, lane, pr, gx, gy);
    if (tid < 64) {
      const int row = tid < 32 ? 0 : HH - 1;
      init_stage_quad<MASK, CSN>(sm, row, lane, pr, gx, y0 - 1 + row);
    } else if (tid < 64 + 2 * TH) {
      const int h = tid - 64;
      const int row = 1 + (h % TH), side = h / TH;
      const int col = side ? 4 + W4 : 3;
      float sn, cs;
      if (CSN) {
        cs = sm.raw[2].v[row][col];
        sn = sm.raw[5].v[row][col];
      } else {
        sincosf(sm.raw[2].v[row][col], &sn, &cs);
      }
      sm.stg[0][row][col] = sm.raw[0].v[row][col];
      sm.stg[1][row][col] = sm.raw[1].v[row][col];
      sm.stg[2][row][col] = cs;
      sm.stg[3][row][col] = sn;
      sm.stg[4][row][col] = sm.raw[3].v[row][col];
      sm.stg[5][row][col] = sm.raw[4].v[row][col];
      const int hy = y0 + row - 1, hx = side ? x0 + W4 : x0 - 1;
      const bool ok = hy < pr.H && hx >= 0 && hx < pr.W;
      sm.stg[6][row][col] = (ok && (!MASK || halo_mask(sm.mk.v, row, side) == 0)) ? 1.f : 0.f;
    }
    __syncthreads();
    if (t + 1 < ch.end) {
      tc = tn;
      issue(tc);
      const int tidn = tile_id(pr, tc);
      hb0 = pr.hbeg[tidn];
      hb1 = pr.hbeg[tidn + 1];
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H) {
      const int c = 4 + 4 * lane;
      float4 O[NSTG_I];
#pragma unroll
      for (int k = 0; k < NSTG_I; ++k) O[k] = lds4(&sm.stg[k][ty + 1][c]);
      const OwnI2 oa = {lo2(O[0]), lo2(O[1]), lo2(O[2]), lo2(O[3]), lo2(O[4]), lo2(O[5])};
      const OwnI2 ob = {hi2(O[0]), hi2(O[1]), hi2(O[2]), hi2(O[3]), hi2(O[4]), hi2(O[5])};
      const float2 z2 = make_float2(0.f, 0.f);
      AccI2 A = {z2, z2, z2, z2, z2, z2}, B = A;
      {
        float L[NSTG_I], R[NSTG_I];
#pragma unroll
        for (int k = 0; k < NSTG_I; ++k) {
          L[k] = __shfl_up_sync(0xffffffffu, O[k].w, 1);
          R[k] = __shfl_down_sync(0xffffffffu, O[k].x, 1);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < NSTG_I; ++k) L[k] = sm.stg[k][ty + 1][3];
        }
        if (lane == 31) {
#pragma unroll
          for (int k = 0; k < NSTG_I; ++k) R[k] = sm.stg[k][ty + 1][4 + W4];
        }
        // A = pixels {0, 2}: left {-1, 1}, right {1, 3} = B
        init_pair2(oa, make_float2(L[0], O[0].z), make_float2(L[1], O[1].z), make_float2(L[2], O[2].z),
                   make_float2(L[3], O[3].z), make_float2(L[4], O[4].z), make_float2(L[5], O[5].z),
                   make_float2(L[6], O[6].z), A);
        init_pair2(oa, ob.dx, ob.dy, ob.c, ob.s, ob.ux, ob.uy, hi2(O[6]), A);
        // B = pixels {1, 3}: left {0, 2} = A, right {2, 4}
        init_pair2(ob, oa.dx, oa.dy, oa.c, oa.s, oa.ux, oa.uy, lo2(O[6]), B);
        init_pair2(ob, make_float2(O[0].y, R[0]), make_float2(O[1].y, R[1]), make_float2(O[2].y, R[2]),
                   make_float2(O[3].y, R[3]), make_float2(O[4].y, R[4]), make_float2(O[5].y, R[5]),
                   make_float2(O[6].y, R[6]), B);
      }
#pragma unroll 1
      for (int dr = 0; dr < 2; ++dr) {
        float4 U[NSTG_I];
        const int row = dr ? ty + 2 : ty;
#pragma unroll
        for (int k = 0; k < NSTG_I; ++k) U[k] = lds4(&sm.stg[k][row][c]);
        init_pair2(oa, lo2(U[0]), lo2(U[1]), lo2(U[2]), lo2(U[3]), lo2(U[4]), lo2(U[5]), lo2(U[6]), A);
        init_pair2(ob, hi2(U[0]), hi2(U[1]), hi2(U[2]), hi2(U[3]), hi2(U[4]), hi2(U[5]), hi2(U[6]), B);
      }
      // scale by w and the own validity, back to plain pixel order
      const float2 wa = mul2(w2, lo2(O[6])), wb = mul2(w2, hi2(O[6]));
      const float2 wa2 = add2(wa, wa), wb2 = add2(wb, wb);
      auto plain = [](float2 a, float2 b) { return make_float4(a.x, b.x, a.y, b.y); };
      const float4 gx4 = plain(mul2(wa, A.gx), mul2(wb, B.gx)), gy4 = plain(mul2(wa, A.gy), mul2(wb, B.gy));
      const float4 gt4 = plain(mul2(wa, A.gt), mul2(wb, B.gt)), dt4 = plain(mul2(wa, A.dt), mul2(wb, B.dt));
      const float4 e4 = plain(mul2(wa, A.e), mul2(wb, B.e)), dd4 = plain(mul2(wa2, A.np), mul2(wb2, B.np));
      float gxv[4] = {gx4.x, gx4.y, gx4.z, gx4.w}, gyv[4] = {gy4.x, gy4.y, gy4.z, gy4.w};
      float gtv[4] = {gt4.x, gt4.y, gt4.z, gt4.w}, dtv[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
      float ev[4] = {e4.x, e4.y, e4.z, e4.w}, ddv[4] = {dd4.x, dd4.y, dd4.z, dd4.w};
      const float vf[4] = {O[6].x, O[6].z, O[6].y, O[6].w};
      const float4 dxp = swz4(O[0]), dyp = swz4(O[1]);
      const long long i = (long long)gy * pr.P + gx;
      for (int h = hcur0; h < hcur1; ++h) {
        const long long k = pr.hpix[h] - i;
        if (k >= 0 && k < 4) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk == k && vf[kk] != 0.f) {
              const float rx = cmp(dxp, kk) - pr.htgt[2 * h], ry = cmp(dyp, kk) - pr.htgt[2 * h + 1];
              gxv[kk] += wfit * rx;
              gyv[kk] += wfit * ry;
              ddv[kk] += wfit;
              ev[kk] += wfit * (rx * rx + ry * ry);
            }
        }
      }
      float md[4], mt[4], cd[4], ct[4], bx[4], by[4], bt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        md[k] = minv_entry(ddv[k], lam, dmin, dmax, pr.use_precond, &cd[k]);
        mt[k] = minv_entry(dtv[k], lam, dmin, dmax, pr.use_precond, &ct[k]);
        bx[k] = -gxv[k];
        by[k] = -gyv[k];
        bt[k] = -gtv[k];
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const float2 md2 = make_float2(md[k], md[k + 1]), mt2 = make_float2(mt[k], mt[k + 1]);
        const float2 bx2 = make_float2(bx[k], bx[k + 1]), by2 = make_float2(by[k], by[k + 1]);
        const float2 bt2 = make_float2(bt[k], bt[k + 1]);
        f2x2_add_prod(acc_rz, bx2, pk_mul(md2, bx2));
        f2x2_add_prod(acc_rz, by2, pk_mul(md2, by2));
        f2x2_add_prod(acc_rz, bt2, pk_mul(mt2, bt2));
        f2x2_add(acc_E, make_float2(ev[k], ev[k + 1]));
      }
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(pr.r + i) = make_float4(bx[0], bx[1], bx[2], bx[3]);
      *reinterpret_cast<float4*>(pr.r + pl + i) = make_float4(by[0], by[1], by[2], by[3]);
      *reinterpret_cast<float4*>(pr.r + 2 * pl + i) = make_float4(bt[0], bt[1], bt[2], bt[3]);
      *reinterpret_cast<float4*>(pr.m + i) = make_float4(md[0], md[1], md[2], md[3]);
      *reinterpret_cast<float4*>(pr.m + pl + i) = make_float4(mt[0], mt[1], mt[2], mt[3]);
      *reinterpret_cast<float4*>(pr.d + i) = z;
      *reinterpret_cast<float4*>(pr.d + pl + i) = z;
      *reinterpret_cast<float4*>(pr.d + 2 * pl + i) = z;
      if (!CSN) {
        *reinterpret_cast<float4*>(pr.csn + i) = swz4(O[2]);
        *reinterpret_cast<float4*>(pr.csn + pl + i) = swz4(O[3]);
      }
      if (pr.lm) {
        *reinterpret_cast<float4*>(pr.dc + i) = make_float4(cd[0], cd[1], cd[2], cd[3]);
        *reinterpret_cast<float4*>(pr.dc + pl + i) = make_float4(ct[0], ct[1], ct[2], ct[3]);
      }
      if (pr.jtf_out) {
        *reinterpret_cast<float4*>(pr.jtf_out + i) = make_float4(gxv[0], gxv[1], gxv[2], gxv[3]);
        *reinterpret_cast<float4*>(pr.jtf_out + pl + i) = make_float4(gyv[0], gyv[1], gyv[2], gyv[3]);
        *reinterpret_cast<float4*>(pr.jtf_out + 2 * pl + i) = make_float4(gtv[0], gtv[1], gtv[2], gtv[3]);
      }
      if (pr.diag_out) {
        *reinterpret_cast<float4*>(pr.diag_out + i) = make_float4(ddv[0], ddv[1], ddv[2], ddv[3]);
        *reinterpret_cast<float4*>(pr.diag_out + pl + i) = make_float4(dtv[0], dtv[1], dtv[2], dtv[3]);
      }
    }
  }
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc_rz), f2x2_fold(acc_E), &s->counter,
                       pr.chunk_end - pr.chunk_begin)) {
    double rz, E;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, rz, E);
    if (threadIdx.x == 0) {
      s->rz = rz;
      s->E = E;
      if (pr.Ehist && k_outer >= 0) pr.Ehist[k_outer] = E;
      s->beta_f = 0.f;
      s->alpha_f = 0.f;         // no step pending (single-reduction PCG)
      s->pcg_active = (rz != 0.0) && isfinite(rz);
      if (!isfinite(rz) || !isfinite(E)) s->nonfinite = 1;
    }
  }
}

#ifndef WARP_INIT_WIDE_MINB
#define WARP_INIT_WIDE_MINB 2       // resident blocks per SM the wide warp PCGInit is compiled for
#endif
// CSN: cos / sin of theta are read from the planes the previous outer
// update wrote (k_grid_step / k_grid_fused_fin with csn_out) instead of being
// evaluated on the tile and its halo; the same bits either way.
template <bool MASK, bool CSN>
__global__ void __launch_bounds__(NT, WARP_INIT_WIDE_MINB) k_warp_init_wide(const GridProb* __restrict__ probs,
    const Chunk* __restrict__ chunks, const int* __restrict__ tiles, double* __restrict__ part, int k_outer,
    float dmin, float dmax) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  InitSmem& sm = *reinterpret_cast<InitSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (tma_ready(pr, &sm)) k_warp_init_wide_body<MASK, CSN>(sm, ch, pr, tiles, part, k_outer, dmin, dmax);
}

// E(x) (mode 0) or E(x + delta) and |F(x) + J(x) delta|^2 (mode 1).
__global__ void __launch_bounds__(NT) k_warp_energy(const GridProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    const int* __restrict__ tiles,
                                                    double* __restrict__ part, int mode,
                                                    int hist_idx) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  __shared__ WarpStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float sw = pr.s_w, sf = pr.s_f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  F2 acc0 = f2_zero(), acc1 = f2_zero();
  const int nsub = pr.tw / TW;
  for (int ts = ch.begin * nsub; ts < ch.end * nsub; ++ts) {
    const int tc = tiles[ts / nsub];
    const int x0 = tile_x0(tc, pr.tw) + TW * (ts % nsub), y0 = tile_y0(tc);
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
      f2_add(acc0, e0);
      f2_add(acc1, e1);
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
  pdl_begin();
  Scalars* s = pr.s;
  if (s->done) return;
  __shared__ PoissonStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  F2 acc_rz = f2_zero(), acc_E = f2_zero();
  const int nsub = pr.tw / TW;
  for (int ts = ch.begin * nsub; ts < ch.end * nsub; ++ts) {
    const int tc = tiles[ts / nsub];
    const int x0 = tile_x0(tc, pr.tw) + TW * (ts % nsub), y0 = tile_y0(tc);
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
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float b = -gr[c];
        pr.r[c * pl + i] = b;
        pr.d[c * pl + i] = 0.f;
        if (pr.jtf_out) pr.jtf_out[c * pl + i] = gr[c];
        f2_add_prod(acc_rz, b, __fmul_rn(mv, b));
      }
      pr.m[i] = mv;
      if (pr.lm) pr.dc[i] = dcv;
      if (pr.diag_out) pr.diag_out[i] = dg;
      f2_add(acc_E, e);
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
  pdl_begin();
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
  F2 acc = f2_zero();
  PoisCell A, B;
  int tc = tiles[ch.begin];
  pois_cell_load(A, pr, pin, tile_x0(tc, 32) + tx, tile_y0(tc) + ty, update, use_beta);
  if (has_halo) pois_cell_load(B, pr, pin, tile_x0(tc, 32) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, 32), y0 = tile_y0(tc);
    const int gx = x0 + tx, gy = y0 + ty;
    const long long i = (long long)gy * P + gx;
    __syncthreads();
    pois_cell_store(st, ty + 1, tx + 1, A, update, use_beta, beta, pout, pl, (gx < W && gy < H) ? i : -1);
    if (has_halo) pois_cell_store(st, hhy, hhx, B, update, use_beta, beta, pout, pl, -1);
    __syncthreads();
    if (t + 1 < ch.end) {
      tc = tiles[t + 1];
      pois_cell_load(A, pr, pin, tile_x0(tc, 32) + tx, tile_y0(tc) + ty, update, use_beta);
      if (has_halo) pois_cell_load(B, pr, pin, tile_x0(tc, 32) - 1 + hhx, tile_y0(tc) - 1 + hhy, update, use_beta);
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
        f2_add_prod(acc, st.p[c][ly][lx], q[c]);
      }
    }
  }
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, pr.chunk_end - pr.chunk_begin)) {
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

// ---------------------------------------------------------------------------
// Wide-tile Poisson kernels (tw = 128).
// Per channel the J^T J row of a free pixel i is q_i = sum_j w_j (p_i - p_j)
// with w_j = 2 for a free neighbour (own + incoming residual), 1 for a fixed
// one (own residual only; p_j = 0 there) and 0 outside the grid, i.e.
// q_i = S_i p_i - sum_j w_j p_j with S_i = sum_j w_j = diag(J^T J)_i.  With
// Y = X - T every residual is r_(i,j) = Y_i - Y_j, so PCGInit is the same
// stencil on Y: J^T F_i = S_i Y_i - sum_j w_j Y_j, E += sum_(j in grid)
// (Y_i - Y_j)^2 over free i.  Quads are held swizzled (pixels 0 2 1 3) so
// that the float2 packs {0, 2} and {1, 3} have their left / right
// neighbours in one register pair.
// ---------------------------------------------------------------------------
constexpr int NRAW_PA = 9;       // r0..r3, M^-1, p_old0..p_old3
constexpr int NRAW_PI = 8;       // X0..X3, T0..T3

// Both wide Poisson kernels keep two tiles in shared memory: while a block
// computes tile t from its raw planes, the copies of tile t + 1 land in the
// other slot (two blocks per SM).  Nothing is staged in between: every thread
// forms the direction (apply) or Y = X - T (PCGInit) of its own quad and of
// the quads above and below it straight from the raw planes, and takes the
// left / right neighbours by warp shuffles (lanes 0 / 31 from the halo
// columns).  Instead of the mask they read the degree plane (one byte per
// pixel, see k_pois_sdeg): S_i + 1 on a free pixel i, S_i = diag(J^T J)_i,
// and 0 on fixed pixels and the row padding.
constexpr int PST = 2;
template <int NR>
struct PoisSlot {
  PlaneT raw[NR];
  BytesT mk;
};
struct PoisWideSmem {
  PoisSlot<NRAW_PA> slot[PST];
  unsigned long long bar[PST];    // tensor-copy completion of each slot
};
struct PoisInitSmem {
  PoisSlot<NRAW_PI> slot[PST];
  unsigned long long bar[PST];
};

// the four degree bytes of the staged quad (row, lane)
__device__ __forceinline__ unsigned int pois_deg4(const unsigned char (*mk)[SPB], int row, int lane) {
  return *reinterpret_cast<const unsigned int*>(&mk[row][16 + 4 * lane]);
}
// degree byte of a halo column (side 0: column -1, side 1: column 128)
__device__ __forceinline__ unsigned int pois_deg_halo(const unsigned char (*mk)[SPB], int row, int side) {
  return halo_mask(mk, row, side);
}
// neighbour weight from its degree byte and whether it lies in the grid: 2
// free, 1 fixed, 0 outside
__device__ __forceinline__ float pois_w(unsigned int deg, bool inb) {
  return inb ? (deg != 0u ? 2.f : 1.f) : 0.f;
}
// weights of the staged quad (row, lane) at (gx, gy), plain order
__device__ __forceinline__ float4 pois_weights(const unsigned char (*mk)[SPB], int row, int lane, const GridProb& pr,
                                               int gx, int gy) {
  const unsigned int d4 = pois_deg4(mk, row, lane);
  const bool iny = gy >= 0 && gy < pr.H;
  return make_float4(pois_w(d4 & 0xffu, iny && gx < pr.W), pois_w((d4 >> 8) & 0xffu, iny && gx + 1 < pr.W),
                     pois_w((d4 >> 16) & 0xffu, iny && gx + 2 < pr.W), pois_w(d4 >> 24, iny && gx + 3 < pr.W));
}
__device__ __forceinline__ float4 free01(const float4& w) {
  return make_float4(w.x > 1.5f ? 1.f : 0.f, w.y > 1.5f ? 1.f : 0.f, w.z > 1.5f ? 1.f : 0.f, w.w > 1.5f ? 1.f : 0.f);
}
// own free flags (1 / 0) and S of the staged quad from its degree bytes, plain order
__device__ __forceinline__ void pois_own(unsigned int d4, float4& fo, float4& S) {
  const float b0 = (float)(d4 & 0xffu), b1 = (float)((d4 >> 8) & 0xffu);
  const float b2 = (float)((d4 >> 16) & 0xffu), b3 = (float)(d4 >> 24);
  fo = make_float4(b0 > 0.f ? 1.f : 0.f, b1 > 0.f ? 1.f : 0.f, b2 > 0.f ? 1.f : 0.f, b3 > 0.f ? 1.f : 0.f);
  S = make_float4(fmaxf(b0 - 1.f, 0.f), fmaxf(b1 - 1.f, 0.f), fmaxf(b2 - 1.f, 0.f), fmaxf(b3 - 1.f, 0.f));
}
__device__ __forceinline__ float4 keep_if(unsigned int d4, const float4& v) {
  return make_float4((d4 & 0xffu) ? v.x : 0.f, (d4 & 0xff00u) ? v.y : 0.f, (d4 & 0xff0000u) ? v.z : 0.f,
                     (d4 & 0xff000000u) ? v.w : 0.f);
}

// Direction of the PCG step on the staged quad (row, c) of one channel, plain
// order: p = M^-1 r + beta p_old with the fused vector update, else the given
// p (raw planes: r0..r3, M^-1, p0..p3).
template <bool UPD>
__device__ __forceinline__ float4 pois_dir4(const PlaneT* raw, int k, int row, int c, const float4& m,
                                            bool use_beta, float2 beta2) {
  if (!UPD) return lds4(&raw[5 + k].v[row][c]);
  float4 v = mul4p(m, lds4(&raw[k].v[row][c]));
  if (use_beta) v = fma4p(beta2, lds4(&raw[5 + k].v[row][c]), v);
  return v;
}
template <bool UPD>
__device__ __forceinline__ float pois_dir1(const PlaneT* raw, int k, int row, int col, bool use_beta,
                                           float beta) {
  if (!UPD) return raw[5 + k].v[row][col];
  float v = raw[4].v[row][col] * raw[k].v[row][col];
  if (use_beta) v = fmaf(beta, raw[5 + k].v[row][col], v);
  return v;
}

// Directions of one staged quad, swizzled (pixels 0 2 1 3).  With the fused
// update they are zero off the free pixels by construction (r and p_old vanish
// there: PCGInit writes r = 0 on every pixel that is not free, the vector
// update keeps it, and the planes start zeroed); a given p (the J^T J p hook)
// is zeroed there from the degree bytes.
template <bool UPD>
__device__ __forceinline__ void pois_dir_quad(const PlaneT* raw, const unsigned char (*mk)[SPB], int row,
                                              int lane, bool use_beta, float2 beta2, float4 (&out)[4]) {
  const int c = 4 + 4 * lane;
  const float4 m = UPD ? lds4(&raw[4].v[row][c]) : make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned int d4 = UPD ? 0u : pois_deg4(mk, row, lane);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = pois_dir4<UPD>(raw, k, row, c, m, use_beta, beta2);
    out[k] = swz4(UPD ? v : keep_if(d4, v));
  }
}

// applyJTJ stencil: with the directions zero off the free pixels, every
// neighbour term w_j p_j is 2 p_j, so per pack and channel
// S p_i - 2 (p_L + (p_R + (p_U + p_D))) (the same roundings as the weighted
// sum: scaling by 2 is exact).  O / U / D swizzled, L / R as in the init.
__device__ __forceinline__ void pois_core_apply(const float4 (&O)[4], const float4 (&U)[4], const float4 (&D)[4],
                                                const float (&L)[4], const float (&R)[4], float2 SA, float2 SB,
                                                float2 (&outA)[4], float2 (&outB)[4]) {
  const float2 two = make_float2(2.f, 2.f);
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    const float2 nA = add2(make_float2(L[ch], O[ch].z), add2(hi2(O[ch]), add2(lo2(U[ch]), lo2(D[ch]))));
    const float2 nB = add2(lo2(O[ch]), add2(make_float2(O[ch].y, R[ch]), add2(hi2(U[ch]), hi2(D[ch]))));
    outA[ch] = sub2(mul2(SA, lo2(O[ch])), mul2(two, nA));
    outB[ch] = sub2(mul2(SB, hi2(O[ch])), mul2(two, nB));
  }
}

// left / right neighbours of the own quad by shuffles (O swizzled: .w is
// pixel 3, .x pixel 0); lanes 0 / 31 leave theirs for the halo columns
template <int N>
__device__ __forceinline__ void pois_side_nbrs(const float4 (&O)[N], float (&L)[N], float (&R)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    L[k] = __shfl_up_sync(0xffffffffu, O[k].w, 1);
    R[k] = __shfl_down_sync(0xffffffffu, O[k].x, 1);
  }
}

// Issues the copies of one Poisson tile: the raw planes and the degree bytes.
template <int NR>
__device__ __forceinline__ void pois_issue(PlaneT* raw, unsigned char (*mk)[SPB], const float* const* src,
                                           const GridProb& pr, int tc, int tid) {
  tile_issue<NR, true>(raw, mk, src, pr.sdeg, pr, tile_x0(tc, W4), tile_y0(tc), tid);
}

// applyJTJ on the thread's own quad of a staged Poisson tile (slot raw / mk;
// i: the quad's pixel index): the direction p = M^-1 r + beta p_old (fused
// update) or the given p on the own quad and its neighbours, q = (J^T J +
// lambda D) p on the free pixels, p and q stored, p.q accumulated.
template <bool UPD>
__device__ __forceinline__ void pois_apply_quad(const PlaneT* raw, const unsigned char (*mk)[SPB],
                                                const GridProb& pr, int ty, int lane, long long i,
                                                bool use_beta, float beta, float2 beta2, float lam,
                                                float* __restrict__ pout, int pl, F2x2& acc) {
  float4 O[4], U[4], D[4];
  float L[4], R[4];
  pois_dir_quad<UPD>(raw, mk, ty + 1, lane, use_beta, beta2, O);
  pois_side_nbrs(O, L, R);
  if (lane == 0) {
    const bool fr = UPD || pois_deg_halo(mk, ty + 1, 0) != 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) L[k] = fr ? pois_dir1<UPD>(raw, k, ty + 1, 3, use_beta, beta) : 0.f;
  }
  if (lane == 31) {
    const bool fr = UPD || pois_deg_halo(mk, ty + 1, 1) != 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) R[k] = fr ? pois_dir1<UPD>(raw, k, ty + 1, 4 + W4, use_beta, beta) : 0.f;
  }
  pois_dir_quad<UPD>(raw, mk, ty, lane, use_beta, beta2, U);
  pois_dir_quad<UPD>(raw, mk, ty + 2, lane, use_beta, beta2, D);
  float4 fo, S;
  pois_own(pois_deg4(mk, ty + 1, lane), fo, S);
  fo = swz4(fo);
  S = swz4(S);
  if (UPD) {
#pragma unroll
    for (int k = 0; k < 4; ++k) *reinterpret_cast<float4*>(pout + k * pl + i) = swz4(O[k]);
  }
  float2 qA[4], qB[4];
  pois_core_apply(O, U, D, L, R, lo2(S), hi2(S), qA, qB);
  float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
  if (pr.lm) dd = swz4(ld4(pr.dc + i));
  const float2 lam2 = make_float2(lam, lam);
  const float2 dA = mul2(lam2, lo2(dd)), dB = mul2(lam2, hi2(dd));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 a = mul2(lo2(fo), fma2(dA, lo2(O[k]), qA[k]));
    const float2 b2 = mul2(hi2(fo), fma2(dB, hi2(O[k]), qB[k]));
    *reinterpret_cast<float4*>(pr.q + k * pl + i) = swz4(cat4(a, b2));
    f2x2_add_prod(acc, lo2(O[k]), a);
    f2x2_add_prod(acc, hi2(O[k]), b2);
  }
}

template <bool UPD>
__device__ __forceinline__ void k_poisson_apply_wide_body(PoisWideSmem& sm, const Chunk& ch, const GridProb& pr,
    const int* __restrict__ tiles, double* __restrict__ part, const float* __restrict__ p_in_override, int par) {
  Scalars* s = pr.s;
  if (s->done || !s->pcg_active) return;
  const int pl = (int)pr.plane;
  const float beta = s->beta_f;
  const float2 beta2 = make_float2(beta, beta);
  const bool use_beta = beta != 0.0f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const float* __restrict__ pin = p_in_override ? p_in_override : pr.p + (long long)(par & 1) * 4 * pl;
  float* __restrict__ pout = pr.p + (long long)((par + 1) & 1) * 4 * pl;
  const float* src[NRAW_PA];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    src[k] = UPD ? pr.r + k * pl : nullptr;
    src[5 + k] = (!UPD || use_beta) ? pin + k * pl : nullptr;
  }
  src[4] = UPD ? pr.m : nullptr;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc = f2x2_zero();
  // tiles arrive by tensor copies (one thread issues them) on the PCG path
  // (the kernel checked tma_ready), by cp.async (every thread) for a caller's p
  constexpr bool tma = UPD;
  // raw planes r0..r3, M^-1, p_old0..p_old3, all in the slab
  auto plane = [&](int k, int& z, int& m) {
    m = 0;
    z = k < 4 ? zslab(pr, 0) + k : k == 4 ? zslab(pr, 1) : (use_beta ? zslab(pr, 2) + (par & 1) * 4 + k - 5 : -1);
  };
  if (tma && tid == 0) {
    mbar_init(&sm.bar[0]);
    mbar_init(&sm.bar[1]);
  }
  __syncthreads();
  auto issue = [&](int slot, int tc) {
    if (tma) {
      if (tid == 0)
        tile_tma<NRAW_PA>(sm.slot[slot].raw, &sm.slot[slot].mk, plane, true, pr, tile_x0(tc, W4), tile_y0(tc),
                          &sm.bar[slot]);
    } else {
      pois_issue<NRAW_PA>(sm.slot[slot].raw, sm.slot[slot].mk.v, src, pr, tc, tid);
    }
  };
  unsigned ph = 0;     // bit b: parity of slot b's next phase
  issue(0, tiles[ch.begin]);
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  for (int t = ch.begin, b = 0; t < ch.end; ++t, b ^= 1) {
    const int tc = tiles[t];
    const int gx = tile_x0(tc, W4) + 4 * lane, gy = tile_y0(tc) + ty;
    const unsigned pb = (ph >> b) & 1u;
    bool ok = true;
    if (tma) {
      ok = mbar_wait(&sm.bar[b], pb);
      ph ^= 1u << b;
    } else {
      cp_async_wait_all();
    }
    // tile t landed; every thread is done with the other slot (tile t - 1)
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar[b], pb);
      return;
    }
    if (t + 1 < ch.end) {
      issue(b ^ 1, tn);
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H)
      pois_apply_quad<UPD>(sm.slot[b].raw, sm.slot[b].mk.v, pr, ty, lane, (long long)gy * pr.P + gx, use_beta, beta,
                           beta2, lam, pout, pl, acc);
  }
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc), f2_zero(), &s->counter, pr.chunk_end - pr.chunk_begin)) {
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

template <bool UPD>
__global__ void __launch_bounds__(NT, 2) k_poisson_apply_wide(const GridProb* __restrict__ probs,
    const Chunk* __restrict__ chunks, const int* __restrict__ tiles, double* __restrict__ part,
    const float* __restrict__ p_in_override, int par) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  PoisWideSmem& sm = *reinterpret_cast<PoisWideSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  // the fused update (the PCG path) stages by tensor copies, a caller's p
  // (the J^T J p hook, UPD = false) by cp.async
  if (!UPD || tma_ready(pr, &sm)) k_poisson_apply_wide_body<UPD>(sm, ch, pr, tiles, part, p_in_override, par);
}

// PCGInit on the thread's own quad of a staged Poisson tile (slot raw / mk):
// J^T F, diag(J^T J), M^-1 and the LM diagonal of the free pixels, r = -J^T F
// and delta = 0 stored, r.z and the energy of the own residuals accumulated.
__device__ __forceinline__ void pois_init_quad(const PlaneT* raw, const unsigned char (*mk)[SPB],
                                               const GridProb& pr, int ty, int lane, int x0, int gx, int gy,
                                               float lam, float dmin, float dmax, int pl,
                                               F2x2& acc_rz, F2x2& acc_E) {
  const int c = 4 + 4 * lane;
  // neighbour weights (swizzled packs: A = pixels {0, 2}, B = {1, 3})
  const float4 wO = swz4(pois_weights(mk, ty + 1, lane, pr, gx, gy));
  const float4 wU = swz4(pois_weights(mk, ty, lane, pr, gx, gy - 1));
  const float4 wD = swz4(pois_weights(mk, ty + 2, lane, pr, gx, gy + 1));
  float wL = __shfl_up_sync(0xffffffffu, wO.w, 1), wR = __shfl_down_sync(0xffffffffu, wO.x, 1);
  if (lane == 0) wL = pois_w(pois_deg_halo(mk, ty + 1, 0), x0 > 0);
  if (lane == 31) wR = pois_w(pois_deg_halo(mk, ty + 1, 1), x0 + W4 < pr.W);
  const float2 waL = make_float2(wL, wO.z), waR = hi2(wO), wbL = lo2(wO), wbR = make_float2(wO.y, wR);
  const float2 waU = lo2(wU), waD = lo2(wD), wbU = hi2(wU), wbD = hi2(wD);
  const float2 SA = add2(add2(waL, waR), add2(waU, waD));
  const float2 SB = add2(add2(wbL, wbR), add2(wbU, wbD));
  const long long i = (long long)gy * pr.P + gx;
  // own pixels free (staged order): free pixels have a non-zero degree byte
  const unsigned int d4 = pois_deg4(mk, ty + 1, lane);
  const float4 fo = swz4(make_float4((d4 & 0xffu) ? 1.f : 0.f, (d4 & 0xff00u) ? 1.f : 0.f,
                                     (d4 & 0xff0000u) ? 1.f : 0.f, (d4 & 0xff000000u) ? 1.f : 0.f));
  // diagonal S on free pixels (0 elsewhere), M^-1, LM damping diagonal
  const float4 dg = swz4(cat4(mul2(lo2(fo), SA), mul2(hi2(fo), SB)));   // plain order
  float4 mv, dcv;
  mv.x = minv_entry(dg.x, lam, dmin, dmax, pr.use_precond, &dcv.x);
  mv.y = minv_entry(dg.y, lam, dmin, dmax, pr.use_precond, &dcv.y);
  mv.z = minv_entry(dg.z, lam, dmin, dmax, pr.use_precond, &dcv.z);
  mv.w = minv_entry(dg.w, lam, dmin, dmax, pr.use_precond, &dcv.w);
  *reinterpret_cast<float4*>(pr.m + i) = mv;
  if (pr.lm) *reinterpret_cast<float4*>(pr.dc + i) = dcv;
  if (pr.diag_out) *reinterpret_cast<float4*>(pr.diag_out + i) = dg;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // per direction (L, R, U, D) and pack: sum over the channels of the own
  // residuals squared (in-grid neighbours only, applied after the loop)
  float2 sa[4], sb[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) sa[d] = sb[d] = make_float2(0.f, 0.f);
  // one channel at a time: J^T F_i = S_i Y_i - sum_j w_j Y_j, with Y = X - T
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 xo = lds4(&raw[k].v[ty + 1][c]), go = lds4(&raw[4 + k].v[ty + 1][c]);
    const float4 O = swz4(cat4(sub2(lo2(xo), lo2(go)), sub2(hi2(xo), hi2(go))));
    const float4 xu = lds4(&raw[k].v[ty][c]), gu = lds4(&raw[4 + k].v[ty][c]);
    const float4 U = swz4(cat4(sub2(lo2(xu), lo2(gu)), sub2(hi2(xu), hi2(gu))));
    const float4 xd = lds4(&raw[k].v[ty + 2][c]), gd = lds4(&raw[4 + k].v[ty + 2][c]);
    const float4 D = swz4(cat4(sub2(lo2(xd), lo2(gd)), sub2(hi2(xd), hi2(gd))));
    float L = __shfl_up_sync(0xffffffffu, O.w, 1), R = __shfl_down_sync(0xffffffffu, O.x, 1);
    if (lane == 0) L = raw[k].v[ty + 1][3] - raw[4 + k].v[ty + 1][3];
    if (lane == 31) R = raw[k].v[ty + 1][4 + W4] - raw[4 + k].v[ty + 1][4 + W4];
    const float2 aL = make_float2(L, O.z), aR = hi2(O), bL = lo2(O), bR = make_float2(O.y, R);
    const float2 aU = lo2(U), aD = lo2(D), bU = hi2(U), bD = hi2(D);
    const float2 nA = fma2(waL, aL, fma2(waR, aR, fma2(waU, aU, mul2(waD, aD))));
    const float2 nB = fma2(wbL, bL, fma2(wbR, bR, fma2(wbU, bU, mul2(wbD, bD))));
    const float2 gA = sub2(mul2(SA, lo2(O)), nA), gB = sub2(mul2(SB, hi2(O)), nB);
    const float4 g = swz4(cat4(mul2(lo2(fo), gA), mul2(hi2(fo), gB)));   // J^T F, plain order
    const float4 bb = make_float4(-g.x, -g.y, -g.z, -g.w);
    *reinterpret_cast<float4*>(pr.r + k * pl + i) = bb;
    *reinterpret_cast<float4*>(pr.d + k * pl + i) = zero;
    if (pr.jtf_out) *reinterpret_cast<float4*>(pr.jtf_out + k * pl + i) = g;
    f2x2_add_prod(acc_rz, lo2(bb), pk_mul(lo2(mv), lo2(bb)));
    f2x2_add_prod(acc_rz, hi2(bb), pk_mul(hi2(mv), hi2(bb)));
    const float2 na[4] = {aL, aR, aU, aD}, nb[4] = {bL, bR, bU, bD};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const float2 da = sub2(lo2(O), na[d]), db = sub2(hi2(O), nb[d]);
      sa[d] = fma2(da, da, sa[d]);
      sb[d] = fma2(db, db, sb[d]);
    }
  }
  // own residuals towards every in-grid neighbour (weight > 0)
  const float2 wa[4] = {waL, waR, waU, waD}, wb[4] = {wbL, wbR, wbU, wbD};
  float2 eA = make_float2(0.f, 0.f), eB = make_float2(0.f, 0.f);
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const float2 ma = make_float2(wa[d].x > 0.5f ? 1.f : 0.f, wa[d].y > 0.5f ? 1.f : 0.f);
    const float2 mb = make_float2(wb[d].x > 0.5f ? 1.f : 0.f, wb[d].y > 0.5f ? 1.f : 0.f);
    eA = fma2(ma, sa[d], eA);
    eB = fma2(mb, sb[d], eB);
  }
  const float2 ea = mul2(lo2(fo), eA), eb = mul2(hi2(fo), eB);
  f2x2_add(acc_E, ea);
  f2x2_add(acc_E, eb);
}

__device__ __forceinline__ void k_poisson_init_wide_body(PoisInitSmem& sm, const Chunk& ch, const GridProb& pr,
    const int* __restrict__ tiles, double* __restrict__ part, int k_outer, float dmin, float dmax) {
  Scalars* s = pr.s;
  if (s->done) return;
  const int pl = (int)pr.plane;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc_rz = f2x2_zero(), acc_E = f2x2_zero();
  // raw planes by tensor copies (the kernel checked tma_ready): X0..X3 (the
  // unknowns), T0..T3 (guidance, in the slab)
  auto plane = [&](int k, int& z, int& m) {
    m = k < 4 ? 1 : 0;
    z = k < 4 ? k : zslab(pr, 4) + k - 4;
  };
  if (tid == 0) {
    mbar_init(&sm.bar[0]);
    mbar_init(&sm.bar[1]);
  }
  __syncthreads();
  auto issue = [&](int slot, int tc) {
    if (tid == 0)
      tile_tma<NRAW_PI>(sm.slot[slot].raw, &sm.slot[slot].mk, plane, true, pr, tile_x0(tc, W4), tile_y0(tc),
                        &sm.bar[slot]);
  };
  unsigned ph = 0;     // bit b: parity of slot b's next phase
  issue(0, tiles[ch.begin]);
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  for (int t = ch.begin, b = 0; t < ch.end; ++t, b ^= 1) {
    const int tc = tiles[t];
    const int x0 = tile_x0(tc, W4), y0 = tile_y0(tc);
    const int gx = x0 + 4 * lane, gy = y0 + ty;
    const unsigned pb = (ph >> b) & 1u;
    const bool ok = mbar_wait(&sm.bar[b], pb);
    ph ^= 1u << b;
    // tile t landed; every thread is done with the other slot (tile t - 1)
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar[b], pb);
      return;
    }
    if (t + 1 < ch.end) {
      issue(b ^ 1, tn);
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H)
      pois_init_quad(sm.slot[b].raw, sm.slot[b].mk.v, pr, ty, lane, x0, gx, gy, lam, dmin, dmax, pl, acc_rz, acc_E);
  }
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc_rz), f2x2_fold(acc_E), &s->counter,
                       pr.chunk_end - pr.chunk_begin)) {
    double rz, E;
    gather_partials(part, pr.chunk_begin, pr.chunk_end, &s->counter, rz, E);
    if (threadIdx.x == 0) {
      s->rz = rz;
      s->E = E;
      if (pr.Ehist && k_outer >= 0) pr.Ehist[k_outer] = E;
      s->beta_f = 0.f;
      s->alpha_f = 0.f;         // no step pending (single-reduction PCG)
      s->pcg_active = (rz != 0.0) && isfinite(rz);
      if (!isfinite(rz) || !isfinite(E)) s->nonfinite = 1;
    }
  }
}

__global__ void __launch_bounds__(NT, 2) k_poisson_init_wide(const GridProb* __restrict__ probs,
    const Chunk* __restrict__ chunks, const int* __restrict__ tiles, double* __restrict__ part, int k_outer,
    float dmin, float dmax) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  PoisInitSmem& sm = *reinterpret_cast<PoisInitSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (tma_ready(pr, &sm)) k_poisson_init_wide_body(sm, ch, pr, tiles, part, k_outer, dmin, dmax);
}

// ---------------------------------------------------------------------------
// Single-reduction PCG iteration of wide Poisson tiles (tw = 128): the
// iteration of k_warp_fused_wide for the four channels of Fig. 27.  z = M^-1 r,
// w = M^-1 q and p are double-buffered; one M^-1 plane serves the four
// channels.  Staged like the warp kernel: tensor copies bring z, w, p_old of
// the tile and its halo into one slot (iteration 0: r and M^-1), phase 2
// forms z = z - alpha w and p = z + beta p_old on every staged quad into a
// staging area (and z, delta += alpha p_old on the own pixels), the next
// tile's copies overlap phase 3, the stencil of k_poisson_apply_wide (the
// directions vanish off the free pixels: q = S p - 2 (p_L + p_R + p_U + p_D)
// per channel, LM damping on the free pixels), w = M^-1 q and the four
// compensated dot products (M^-1 of the own pixels from the degree bytes
// under Gauss-Newton).  Per pixel of an active tile: read z, w, p_old 48,
// degree byte 1, M^-1 4 (LM), delta 16; write z, w, p, delta 64 = 133 B (GN:
// 129 B; two-pass: 69 + 100 B).
// ---------------------------------------------------------------------------
constexpr int NRAW_PF = 12;      // z0..z3 w0..w3 p0..p3 (iteration 0: r0..r3 at 0..3, M^-1 at 4)
constexpr int NSTG_PF = 4;       // p0..p3, each quad stored as pixels 0 2 1 3

struct PoisFusedSmem {
  PlaneT raw[NRAW_PF];
  float stg[NSTG_PF][HH][SP];    // halo columns -1 / 128 live at 3 / 132, in plain order
  BytesT mk[2];                  // degree bytes of the current / next tile
  unsigned long long bar;
};

__device__ __forceinline__ void pois_fused_body(PoisFusedSmem& sm, const Chunk& ch, const GridProb& pr,
                                                const int* __restrict__ tiles, double* __restrict__ part, int it) {
  Scalars* s = pr.s;
  if (s->done) return;
  const int first = it == 0;
  const float alpha = first ? 0.f : s->alpha_f;
  const long long pl = pr.plane;
  const float* __restrict__ pin = pr.p + (long long)(it & 1) * 4 * pl;
  if (!s->pcg_active) {
    if (alpha != 0.f) fused_pending<4>(ch, pr, tiles, part, pin, alpha);
    return;
  }
  const float beta = first ? 0.f : s->beta_f;
  const int use_beta = beta != 0.0f;
  const float lam = pr.lm ? s->lambda_f : 0.0f;
  float* __restrict__ pout = pr.p + (long long)((it + 1) & 1) * 4 * pl;
  float* __restrict__ zout = pr.zb + (long long)((it + 1) & 1) * 4 * pl;
  float* __restrict__ wout = pr.wb + (long long)((it + 1) & 1) * 4 * pl;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  F2x2 acc_pq = f2x2_zero(), acc_qz = f2x2_zero(), acc_qw = f2x2_zero(), acc_zr = f2x2_zero();
  const int zz = pr.zpack2 & 63, zw = (pr.zpack2 >> 6) & 63, par4 = (it & 1) * 4;
  // raw planes, all in the slab (tensor map 0); the degree bytes by map 2
  auto plane = [&](int k, int& z, int& m) {
    m = 0;
    if (first)
      z = k < 4 ? zslab(pr, 0) + k : k == 4 ? zslab(pr, 1) : -1;
    else
      z = k < 4 ? zz + par4 + k : k < 8 ? zw + par4 + k - 4 : zslab(pr, 2) + par4 + k - 8;
  };
  auto issue = [&](int tcx, int slot) {
    if (tid == 0) tile_tma<NRAW_PF>(sm.raw, &sm.mk[slot], plane, true, pr, tile_x0(tcx, W4), tile_y0(tcx), &sm.bar);
  };
  float4 dl[4];       // delta of the own pixels, loaded before the staging wait
  auto stage = [&](int row, bool own, long long i) {
    const int c = 4 + 4 * lane;
    auto R = [&](int k) { return lds4(&sm.raw[k].v[row][c]); };
    const float4 m = first ? R(4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 z = first ? mul4s(m, R(k)) : fma4s(-alpha, R(4 + k), R(k));
      const float4 p = use_beta ? fma4s(beta, R(8 + k), z) : z;
      sts4(&sm.stg[k][row][c], swz4(p));
      if (own) {
        *reinterpret_cast<float4*>(zout + k * pl + i) = z;
        if (!first) *reinterpret_cast<float4*>(pr.d + k * pl + i) = fma4s(alpha, R(8 + k), dl[k]);
      }
    }
  };
  int tc = tiles[ch.begin];
  int tn = ch.begin + 1 < ch.end ? tiles[ch.begin + 1] : 0;
  unsigned phase = 0;
  int slot = 0;
  issue(tc, 0);
  for (int t = ch.begin; t < ch.end; ++t) {
    const int x0 = tile_x0(tc, W4), y0 = tile_y0(tc);
    const int gx = x0 + 4 * lane, gy = y0 + ty;
    const long long i = (long long)gy * pr.P + gx;
    if (!first && gy < pr.H) {
#pragma unroll
      for (int k = 0; k < 4; ++k) dl[k] = *reinterpret_cast<const float4*>(pr.d + k * pl + i);
    }
    const unsigned pb = phase;
    const bool ok = mbar_wait(&sm.bar, pb);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      staging_timeout(s, &sm.bar, pb);
      return;
    }
    const unsigned char (*mk)[SPB] = sm.mk[slot].v;
    // phase 2: z and the direction on the tile and its halo
    stage(ty + 1, gy < pr.H, i);
    if (tid < 64) {
      stage(tid < 32 ? 0 : HH - 1, false, 0);
    } else if (tid < 64 + 2 * TH) {
      const int h = tid - 64;
      const int row = 1 + (h % TH), side = h / TH;
      const int col = side ? 4 + W4 : 3;
      auto R = [&](int k) { return sm.raw[k].v[row][col]; };
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float z = first ? __fmul_rn(R(4), R(k)) : __fmaf_rn(-alpha, R(4 + k), R(k));
        if (use_beta) z = __fmaf_rn(beta, R(8 + k), z);
        sm.stg[k][row][col] = z;
      }
    }
    __syncthreads();
    // the raw buffer is free: start the next tile's copies
    if (t + 1 < ch.end) {
      tc = tn;
      issue(tc, slot ^ 1);
      if (t + 2 < ch.end) tn = tiles[t + 2];
    }
    if (gy < pr.H) {                          // warp-uniform: one warp per row
      const int c = 4 + 4 * lane;
      float4 O[4], U[4], D[4];
      float L[4], R[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        O[k] = lds4(&sm.stg[k][ty + 1][c]);
        *reinterpret_cast<float4*>(pout + k * pl + i) = swz4(O[k]);
      }
      pois_side_nbrs(O, L, R);
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) L[k] = sm.stg[k][ty + 1][3];
      }
      if (lane == 31) {
#pragma unroll
        for (int k = 0; k < 4; ++k) R[k] = sm.stg[k][ty + 1][4 + W4];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        U[k] = lds4(&sm.stg[k][ty][c]);
        D[k] = lds4(&sm.stg[k][ty + 2][c]);
      }
      float4 fo, S;
      pois_own(pois_deg4(mk, ty + 1, lane), fo, S);
      fo = swz4(fo);
      S = swz4(S);
      float2 qA[4], qB[4];
      pois_core_apply(O, U, D, L, R, lo2(S), hi2(S), qA, qB);
      float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
      if (pr.lm) dd = swz4(ld4(pr.dc + i));
      const float2 lam2 = make_float2(lam, lam);
      const float2 dA = mul2(lam2, lo2(dd)), dB = mul2(lam2, hi2(dd));
      // w = M^-1 q and the four inner products (swizzled packs: A = pixels
      // {0, 2}, B = {1, 3}); z of the own pixels comes back from the stores
      // of phase 2 (this thread's own writes).  Under Gauss-Newton M^-1 and
      // the diagonal (r = diag z) follow from the degree bytes: diag = S, M^-1
      // = 1 / S, the values PCGInit wrote (1 where S = 0 or without the
      // preconditioner); under LM the damping enters, so M^-1 is read.
      float4 ms, rc;
      if (!pr.lm) {
        auto inv = [&](float v) { return pr.use_precond && v > 0.f ? __frcp_rn(v) : 1.f; };
        auto dg = [&](float v) { return pr.use_precond && v > 0.f ? v : 1.f; };
        ms = make_float4(inv(S.x), inv(S.y), inv(S.z), inv(S.w));
        rc = make_float4(dg(S.x), dg(S.y), dg(S.z), dg(S.w));
      } else {
        ms = swz4(ld4(pr.m + i));
        rc = rcp4(ms);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 a = mul2(lo2(fo), fma2(dA, lo2(O[k]), qA[k]));
        const float2 b2 = mul2(hi2(fo), fma2(dB, hi2(O[k]), qB[k]));
        const float2 wa = mul2(lo2(ms), a), wb = mul2(hi2(ms), b2);
        *reinterpret_cast<float4*>(wout + k * pl + i) = swz4(cat4(wa, wb));
        const float4 zs = swz4(*reinterpret_cast<const float4*>(zout + k * pl + i));
        const float2 ra = mul2(lo2(rc), lo2(zs)), rb = mul2(hi2(rc), hi2(zs));
        f2x2_add_prod(acc_pq, lo2(O[k]), a);
        f2x2_add_prod(acc_pq, hi2(O[k]), b2);
        f2x2_add_prod(acc_qw, wa, a);
        f2x2_add_prod(acc_qw, wb, b2);
        f2x2_add_prod(acc_qz, lo2(zs), a);
        f2x2_add_prod(acc_qz, hi2(zs), b2);
        f2x2_add_prod(acc_zr, lo2(zs), ra);
        f2x2_add_prod(acc_zr, hi2(zs), rb);
      }
    }
    slot ^= 1;
  }
  fused_finish(pr, part, acc_pq, acc_qz, acc_qw, acc_zr);
}

__global__ void __launch_bounds__(NT, 2) k_poisson_fused_wide(const GridProb* __restrict__ probs,
                                                              const Chunk* __restrict__ chunks,
                                                              const int* __restrict__ tiles,
                                                              double* __restrict__ part, int it) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  PoisFusedSmem& sm = *reinterpret_cast<PoisFusedSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (threadIdx.x == 0) mbar_init(&sm.bar);
  __syncthreads();
  if (tma_ready(pr, &sm)) pois_fused_body(sm, ch, pr, tiles, part, it);
}

// Degree plane of a wide Poisson problem: S_i + 1 on a free pixel i, where
// S_i = diag(J^T J)_i sums 2 per free and 1 per fixed in-grid neighbour
// (Fig. 27: each free pixel owns one residual per in-grid neighbour, a free
// neighbour adds its own residual towards i); 0 on fixed pixels and on the
// row padding.
__global__ void k_pois_sdeg(int W, int H, int P, const uint8_t* __restrict__ mask, uint8_t* __restrict__ out) {
  const long long n = (long long)P * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / P), x = (int)(i % P);
    unsigned int v = 0;
    if (x < W && (!mask || mask[i] == 0)) {
      unsigned int S = 0;
      const int nx[4] = {x - 1, x + 1, x, x}, ny[4] = {y, y, y - 1, y + 1};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (nx[k] >= 0 && nx[k] < W && ny[k] >= 0 && ny[k] < H)
          S += (!mask || mask[(long long)ny[k] * P + nx[k]] == 0) ? 2u : 1u;
      v = S + 1;
    }
    out[i] = (uint8_t)v;
  }
}

__global__ void __launch_bounds__(NT) k_poisson_energy(const GridProb* __restrict__ probs,
                                                       const Chunk* __restrict__ chunks,
                                                       const int* __restrict__ tiles,
                                                       double* __restrict__ part, int mode,
                                                       int hist_idx) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  Scalars* s = pr.s;
  if (mode == 1 && s->done) return;
  __shared__ PoissonStage st;
  const long long pl = pr.plane;
  const int P = pr.P, W = pr.W, H = pr.H;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  F2 acc0 = f2_zero(), acc1 = f2_zero();
  const int nsub = pr.tw / TW;
  for (int ts = ch.begin * nsub; ts < ch.end * nsub; ++ts) {
    const int tc = tiles[ts / nsub];
    const int x0 = tile_x0(tc, pr.tw) + TW * (ts % nsub), y0 = tile_y0(tc);
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
      f2_add(acc0, e0);
      f2_add(acc1, e0);
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
// One vector-update pass of the block's chunk (shared by the per-step kernel
// and the persistent PCG kernel).  p and q were written earlier in the same
// persistent launch, so they are read through L2 (ld.global.cg), not the
// read-only path.
template <int NX>
__device__ __forceinline__ void update_body(const Chunk& ch, const GridProb& pr, const int* __restrict__ tiles,
                                            double* __restrict__ part, int par) {
  constexpr int NM = NX == 3 ? 2 : 1;
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
  F2x2 acc = f2x2_zero();
  const int qrow = pr.tw / 4;        // float4 quads per tile row
  const int QPT = qrow * TH;         // float4 quads per tile
  const int nq = (ch.end - ch.begin) * QPT;
  // the tile index of the thread's next quad is loaded one step ahead
  int tc_next = threadIdx.x < nq ? tiles[ch.begin + threadIdx.x / QPT] : 0;
  for (int k = threadIdx.x; k < nq; k += NT) {
    const int tc = tc_next;
    if (k + NT < nq) tc_next = tiles[ch.begin + (k + NT) / QPT];
    const int w = k % QPT;
    const int y = tile_y0(tc) + w / qrow;
    if (y >= pr.H) continue;
    // Poisson, 128-pixel tiles: a quad without a free pixel keeps zero
    // delta, r, p and q, so it is skipped
    if (NX == 4 && pr.live && !((__ldg(pr.live + (long long)y * pr.ntx + (tc & 0xffff)) >> (w % qrow)) & 1u)) continue;
    const long long j = (long long)y * P4 + tile_x0(tc, pr.tw) / 4 + w % qrow;
    float4 pv[NX], qv[NX], dv[NX], rv[NX], mv[NM];
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      pv[c] = __ldcg(pn + c * pl4 + j);
      qv[c] = __ldcg(q4 + c * pl4 + j);
      dv[c] = d4[c * pl4 + j];
      rv[c] = r4[c * pl4 + j];
    }
#pragma unroll
    for (int c = 0; c < NM; ++c) mv[c] = __ldg(m4 + c * pl4 + j);
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      // distinct-diagonal plane: warp (x, y) -> 0, theta -> 1; Poisson -> 0
      const float4 m = mv[NX == 3 ? (c == 2 ? 1 : 0) : 0];
      // explicit roundings: the same bits in every kernel using this body
      dv[c].x = __fmaf_rn(alpha, pv[c].x, dv[c].x); dv[c].y = __fmaf_rn(alpha, pv[c].y, dv[c].y);
      dv[c].z = __fmaf_rn(alpha, pv[c].z, dv[c].z); dv[c].w = __fmaf_rn(alpha, pv[c].w, dv[c].w);
      rv[c].x = __fmaf_rn(-alpha, qv[c].x, rv[c].x); rv[c].y = __fmaf_rn(-alpha, qv[c].y, rv[c].y);
      rv[c].z = __fmaf_rn(-alpha, qv[c].z, rv[c].z); rv[c].w = __fmaf_rn(-alpha, qv[c].w, rv[c].w);
      f2x2_add_prod(acc, lo2(rv[c]), pk_mul(lo2(m), lo2(rv[c])));
      f2x2_add_prod(acc, hi2(rv[c]), pk_mul(hi2(m), hi2(rv[c])));
      d4[c * pl4 + j] = dv[c];
      r4[c * pl4 + j] = rv[c];
    }
  }
  if (publish_partials(part, blockIdx.x, f2x2_fold(acc), f2_zero(), &s->counter, pr.chunk_end - pr.chunk_begin)) {
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
__global__ void __launch_bounds__(NT) k_grid_update(const GridProb* __restrict__ probs,
                                                    const Chunk* __restrict__ chunks,
                                                    const int* __restrict__ tiles,
                                                    double* __restrict__ part, int par) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  update_body<NX>(ch, pr, tiles, part, par);
}

// Persistent PCG loop of the wide warp (tw = 128): n_inner iterations of
// applyJTJ + vector update in one cooperative launch (every block resident),
// separated by grid-wide barriers instead of kernel boundaries.  Block b
// keeps chunk b for the whole loop, so the reductions are the same as those
// of the per-step kernels.  A barrier that times out ends the launch early
// with the barrier's timeout flag set.
template <bool MASK>
__global__ void __launch_bounds__(NT, 2) k_warp_pcg_coop(const GridProb* __restrict__ probs,
                                                         const Chunk* __restrict__ chunks,
                                                         const int* __restrict__ tiles,
                                                         double* __restrict__ part, GridBarrier* gb,
                                                         int par0, int n_inner) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  WideSmem& sm = *reinterpret_cast<WideSmem*>(dyn_smem);
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  if (threadIdx.x == 0) mbar_init(&sm.bar);
  __syncthreads();
  unsigned phase = 0;
  const bool tma = wide_tma(pr, &sm);
  for (int it = 0; it < n_inner; ++it) {
    if (tma)
      apply_wide_body<MASK, true>(sm, ch, pr, tiles, part, nullptr, par0 + it, 1, phase);
    else
      apply_wide_body<MASK, false>(sm, ch, pr, tiles, part, nullptr, par0 + it, 1, phase);
    if (!grid_sync(gb, gridDim.x)) return;
    update_body<3>(ch, pr, tiles, part, par0 + it);
    if (it + 1 < n_inner && !grid_sync(gb, gridDim.x)) return;
  }
}

// x += delta over the owned pixels (cond: 0 always, 1 only if s->accept);
// csn_out (wide warps): also cos / sin of the new theta.
template <int NX>
__global__ void __launch_bounds__(NT) k_grid_step(const GridProb* __restrict__ probs,
                                                  const Chunk* __restrict__ chunks,
                                                  const int* __restrict__ tiles, int cond, int csn_out) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (cond && !pr.s->accept) return;
  if (!cond && pr.s->done) return;
  const long long pl = pr.plane;
  float* __restrict__ x = pr.x;
  const float* __restrict__ d = pr.d;
  const bool csn = NX == 3 && csn_out && pr.csn;
  // float4 quads of the chunk's tiles; the pitched padding columns hold zeros
  // in both planes, so only rows past H are skipped
  const int qrow = pr.tw / 4, qpt = qrow * TH;
  const int nq = (ch.end - ch.begin) * qpt;
  for (int u = threadIdx.x; u < nq; u += NT) {
    const int tc = tiles[ch.begin + u / qpt];
    const int q = u % qpt;
    const int gy = tile_y0(tc) + q / qrow;
    if (gy >= pr.H) continue;
    const long long i = (long long)gy * pr.P + tile_x0(tc, pr.tw) + 4 * (q % qrow);
    float4 xv[NX], dv[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      xv[c] = *reinterpret_cast<const float4*>(x + c * pl + i);
      dv[c] = __ldg(reinterpret_cast<const float4*>(d + c * pl + i));
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      xv[c] = make_float4(xv[c].x + dv[c].x, xv[c].y + dv[c].y, xv[c].z + dv[c].z, xv[c].w + dv[c].w);
      *reinterpret_cast<float4*>(x + c * pl + i) = xv[c];
    }
    if (csn) store_csn(pr, i, xv[2]);
  }
}

// cos / sin of theta at the current unknowns (wide warps; before a PCGInit
// that reads them when no outer update wrote them)
__global__ void __launch_bounds__(NT) k_warp_csn(const GridProb* __restrict__ probs, const Chunk* __restrict__ chunks,
                                                 const int* __restrict__ tiles) {
  const Chunk ch = chunks[blockIdx.x];
  const GridProb pr = probs[ch.prob];
  pdl_begin();
  if (!pr.csn) return;
  const int qrow = W4 / 4, qpt = qrow * TH;
  const int nq = (ch.end - ch.begin) * qpt;
  for (int u = threadIdx.x; u < nq; u += NT) {
    const int tc = tiles[ch.begin + u / qpt];
    const int q = u % qpt;
    const int gy = tile_y0(tc) + q / qrow;
    if (gy >= pr.H) continue;
    const long long i = (long long)gy * pr.P + tile_x0(tc, W4) + 4 * (q % qrow);
    store_csn(pr, i, *reinterpret_cast<const float4*>(pr.x + 2 * pr.plane + i));
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t grid_kernels_prepare() {
  static cudaError_t status = cudaErrorNotReady;
  static std::once_flag once;
  std::call_once(once, [] {
    const int bytes = (int)sizeof(WideSmem);
    cudaError_t e = cudaFuncSetAttribute(k_warp_apply_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_apply_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_apply_wide<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_apply_wide<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    const int ibytes = (int)sizeof(InitSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ibytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ibytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ibytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ibytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_init_wide<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    const int pbytes = (int)sizeof(PoisWideSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_poisson_apply_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pbytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_poisson_apply_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, pbytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_poisson_init_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(PoisInitSmem));
    const int fbytes = (int)sizeof(FusedSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_fused_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fbytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_fused_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fbytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_fused_wide<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_fused_wide<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_poisson_fused_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(PoisFusedSmem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_pcg_coop<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_pcg_coop<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_pcg_coop<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_warp_pcg_coop<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    status = e;
  });
  return status;
}

void launch_grid_init(int kind, const GridLaunch& L, int k_outer, float dmin, float dmax, int csn_in) {
  if (kind == K_WARP && L.tw == 128) {
    auto k = L.masked ? (csn_in ? k_warp_init_wide<true, true> : k_warp_init_wide<true, false>)
                      : (csn_in ? k_warp_init_wide<false, true> : k_warp_init_wide<false, false>);
    launch_pdl(k, L.nchunks, NT, sizeof(InitSmem), L.stream, L.probs, L.chunks, L.tiles, L.part, k_outer, dmin, dmax);
  } else if (kind == K_WARP) {
    launch_pdl(k_warp_init, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, k_outer, dmin, dmax);
  } else if (L.tw == W4) {
    launch_pdl(k_poisson_init_wide, L.nchunks, NT, sizeof(PoisInitSmem), L.stream, L.probs, L.chunks, L.tiles,
               L.part, k_outer, dmin, dmax);
  } else {
    launch_pdl(k_poisson_init, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, k_outer, dmin, dmax);
  }
}

void launch_grid_apply(int kind, const GridLaunch& L, const float* p_override, int par, int update) {
  if (kind == K_WARP && L.tw == 128 && L.masked)
    launch_pdl(k_warp_apply_wide<true>, L.nchunks, NT, sizeof(WideSmem), L.stream, L.probs, L.chunks, L.tiles, L.part,
                                                                         p_override, par, update);
  else if (kind == K_WARP && L.tw == 128)
    launch_pdl(k_warp_apply_wide<false>, L.nchunks, NT, sizeof(WideSmem), L.stream, L.probs, L.chunks, L.tiles, L.part,
                                                                          p_override, par, update);
  else if (kind == K_WARP)
    launch_pdl(k_warp_apply, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, p_override, par, update);
  else
    if (L.tw == W4 && update)
      launch_pdl(k_poisson_apply_wide<true>, L.nchunks, NT, sizeof(PoisWideSmem), L.stream, L.probs, L.chunks,
                 L.tiles, L.part, p_override, par);
    else if (L.tw == W4)
      launch_pdl(k_poisson_apply_wide<false>, L.nchunks, NT, sizeof(PoisWideSmem), L.stream, L.probs, L.chunks,
                 L.tiles, L.part, p_override, par);
    else
      launch_pdl(k_poisson_apply, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, p_override, par,
                 update);
}

void launch_grid_update(int kind, const GridLaunch& L, int par) {
  if (kind == K_WARP)
    launch_pdl(k_grid_update<3>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, par);
  else
    launch_pdl(k_grid_update<4>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, par);
}

void launch_grid_fused(int kind, const GridLaunch& L, int it) {
  if (kind == K_POISSON)
    launch_pdl(k_poisson_fused_wide, L.nchunks, NT, sizeof(PoisFusedSmem), L.stream, L.probs, L.chunks, L.tiles,
               L.part, it);
  else if (L.masked)
    launch_pdl(k_warp_fused_wide<true>, L.nchunks, NT, sizeof(FusedSmem), L.stream, L.probs, L.chunks, L.tiles,
               L.part, it);
  else
    launch_pdl(k_warp_fused_wide<false>, L.nchunks, NT, sizeof(FusedSmem), L.stream, L.probs, L.chunks, L.tiles,
               L.part, it);
}

void launch_grid_fused_fin(int kind, const GridLaunch& L, int par, int step, int csn_out) {
  if (kind == K_POISSON)
    launch_pdl(k_grid_fused_fin<4>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, par, step, 0);
  else
    launch_pdl(k_grid_fused_fin<3>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, par, step, csn_out);
}

void launch_grid_csn(const GridLaunch& L) {
  launch_pdl(k_warp_csn, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles);
}

void launch_grid_energy(int kind, const GridLaunch& L, int mode, int hist_idx) {
  if (kind == K_WARP)
    launch_pdl(k_warp_energy, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, mode, hist_idx);
  else
    launch_pdl(k_poisson_energy, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, L.part, mode, hist_idx);
}

void launch_pois_sdeg(int W, int H, int P, const uint8_t* mask, uint8_t* out, cudaStream_t st) {
  const long long n = (long long)P * H;
  const int blocks = (int)std::min<long long>((n + NT - 1) / NT, 152LL * 16);
  k_pois_sdeg<<<blocks, NT, 0, st>>>(W, H, P, mask, out);
}

void launch_grid_step(int kind, const GridLaunch& L, int cond, int csn_out) {
  if (kind == K_WARP)
    launch_pdl(k_grid_step<3>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, cond, csn_out);
  else
    launch_pdl(k_grid_step<4>, L.nchunks, NT, 0, L.stream, L.probs, L.chunks, L.tiles, cond, 0);
}

int grid_coop_capacity(int masked) {
  if (grid_kernels_prepare() != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = masked ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_pcg_coop<true>, NT,
                                                                          sizeof(WideSmem))
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_pcg_coop<false>, NT,
                                                                          sizeof(WideSmem));
  return e == cudaSuccess ? per_sm * sms : 0;
}

cudaError_t launch_grid_pcg_coop(const GridLaunch& L, GridBarrier* gb, int par0, int n_inner) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.nchunks);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(WideSmem);
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return L.masked ? cudaLaunchKernelEx(&cfg, k_warp_pcg_coop<true>, L.probs, L.chunks, L.tiles, L.part, gb, par0,
                                       n_inner)
                  : cudaLaunchKernelEx(&cfg, k_warp_pcg_coop<false>, L.probs, L.chunks, L.tiles, L.part, gb, par0,
                                       n_inner);
}

// Barrier self-test: `rounds` barriers among gridDim.x blocks that await
// `expected` arrivals each; a block that times out stops.
__global__ void k_barrier_selftest(GridBarrier* gb, unsigned int expected, int rounds,
                                   unsigned long long limit_ns) {
  for (int r = 0; r < rounds; ++r)
    if (!grid_sync(gb, expected, limit_ns)) return;
}

// Self-test of the bounded staging wait: complete = 1 arrives on the
// mbarrier (no bytes expected), so the phase completes; complete = 0 leaves
// it pending, so every thread's wait runs out after limit_ns.  *out = 1 if
// any wait ran out.
__global__ void k_staging_selftest(int complete, unsigned long long limit_ns, int* out) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  if (complete && threadIdx.x == 0) mbar_expect(&bar, 0u);
  const bool ok = mbar_wait(&bar, 0u, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) *out = 1;
}

cudaError_t launch_staging_selftest(int complete, unsigned long long limit_ns, int* out, cudaStream_t st) {
  k_staging_selftest<<<2, NT, 0, st>>>(complete, limit_ns, out);
  return cudaGetLastError();
}

cudaError_t launch_barrier_selftest(GridBarrier* gb, int nblocks, unsigned int expected, int rounds,
                                    unsigned long long limit_ns, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(NT);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_selftest, gb, expected, rounds, limit_ns);
}

}  // namespace optgb
