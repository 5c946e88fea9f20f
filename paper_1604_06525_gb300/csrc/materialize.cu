// Materialized-Jacobian variant of applyJTJ (Sec. 7 "Matrix-free vs.
// Materialized", Sec. 8.3 / Fig. 16; the paper materializes J with evalJ and
// runs its sparse products with a library; here both products are
// hand-written).
//
// Structure (built once per problem on the host): J in CSR, one row per
// residual component, columns in the internal unknown index space
// (component * plane + pixel / vertex); J^T in CSR over the unknown columns
// that have at least one entry, with the permutation that gathers J's values
// into J^T's order.  Values: evalJ refreshes the entries that depend on x once
// per outer iteration (warp: the rotation column; mesh: the three angle
// columns; Poisson's J is constant), then the permutation fills J^T.
//
// Per PCG iteration: direction update p = M^-1 r + beta p over the non-empty
// unknowns, t = J p (one thread per row), q = J^T t + lambda D p with a
// float64 p.q reduction (one thread per unknown), then the shared vector
// update of the matrix-free path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"
#include "opt_launch.h"
#include "opt_problem.h"

namespace optgb {

namespace {

struct CompMap {
  int mp[6];   // distinct-diagonal plane of each unknown component
};

__global__ void __launch_bounds__(NT) k_evalj_warp(int G, const int* __restrict__ col, float* __restrict__ val,
                                                   const float* __restrict__ x, const float* __restrict__ U,
                                                   long long pl, float sw, const Scalars* __restrict__ s) {
  if (s->done) return;
  for (int g = blockIdx.x * NT + threadIdx.x; g < G; g += gridDim.x * NT) {
    const int i = col[6 * g], j = col[6 * g + 1];
    float sn, cs;
    sincosf(x[2 * pl + i], &sn, &cs);
    const float vx = U[i] - U[j], vy = U[pl + i] - U[pl + j];
    const float gx = -sw * (-sn * vx - cs * vy), gy = -sw * (cs * vx - sn * vy);
    float* v = val + 6 * (long long)g;
    v[0] = sw; v[1] = -sw; v[2] = gx;
    v[3] = sw; v[4] = -sw; v[5] = gy;
  }
}

__global__ void __launch_bounds__(NT) k_evalj_mesh(int E, const int* __restrict__ e0, const int* __restrict__ e1,
                                                   float* __restrict__ val, const float* __restrict__ x,
                                                   const float* __restrict__ U, long long pl, float sw,
                                                   const Scalars* __restrict__ s) {
  if (s->done) return;
  for (int e = blockIdx.x * NT + threadIdx.x; e < E; e += gridDim.x * NT) {
    const int a = e0[e], b = e1[e];
    const RotV R = rot_apply(x[3 * pl + a], x[4 * pl + a], x[5 * pl + a], U[a] - U[b],
                             U[pl + a] - U[pl + b], U[2 * pl + a] - U[2 * pl + b]);
    float* v = val + 15 * (long long)e;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[5 * c] = sw;
      v[5 * c + 1] = -sw;
      v[5 * c + 2] = -sw * R.g[0][c];
      v[5 * c + 3] = -sw * R.g[1][c];
      v[5 * c + 4] = -sw * R.g[2][c];
    }
  }
}

__global__ void __launch_bounds__(NT) k_gather_vals(long long nnz, const int* __restrict__ perm,
                                                    const float* __restrict__ val, float* __restrict__ tval,
                                                    const Scalars* __restrict__ s) {
  if (s->done) return;
  for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < nnz; k += (long long)gridDim.x * NT)
    tval[k] = val[perm[k]];
}

// p = M^-1 r + beta p_old over the non-empty unknowns.
__global__ void __launch_bounds__(NT) k_csr_direction(int nT, const int* __restrict__ t_unk, long long pl,
                                                      CompMap cm, const float* __restrict__ m,
                                                      const float* __restrict__ r, const float* __restrict__ pin,
                                                      float* __restrict__ pout, const Scalars* __restrict__ s) {
  if (s->done || !s->pcg_active) return;
  const float beta = s->beta_f;
  for (int k = blockIdx.x * NT + threadIdx.x; k < nT; k += gridDim.x * NT) {
    const int u = t_unk[k];
    const int c = (int)(u / pl);
    const long long idx = u - c * pl;
    float v = m[cm.mp[c] * pl + idx] * r[u];
    if (beta != 0.0f) v += beta * pin[u];
    pout[u] = v;
  }
}

// t = J p, one thread per residual row.
__global__ void __launch_bounds__(NT) k_csr_jp(int R, const int* __restrict__ rp, const int* __restrict__ col,
                                               const float* __restrict__ val, const float* __restrict__ p,
                                               float* __restrict__ t, const Scalars* __restrict__ s) {
  if (s->done || !s->pcg_active) return;
  for (int row = blockIdx.x * NT + threadIdx.x; row < R; row += gridDim.x * NT) {
    float acc = 0.f;
    for (int k = rp[row]; k < rp[row + 1]; ++k) acc += val[k] * p[col[k]];
    t[row] = acc;
  }
}

// q = J^T t (+ lambda D p), one thread per non-empty unknown; float64 p.q -> alpha.
__global__ void __launch_bounds__(NT) k_csr_jtt(int nT, const int* __restrict__ t_unk, const int* __restrict__ t_ptr,
                                                const int* __restrict__ t_row, const float* __restrict__ t_val,
                                                const float* __restrict__ t, const float* __restrict__ p,
                                                float* __restrict__ q, const float* __restrict__ dc, int lm,
                                                long long pl, CompMap cm, Scalars* __restrict__ s,
                                                double* __restrict__ part) {
  if (s->done || !s->pcg_active) return;
  const float lam = lm ? s->lambda_f : 0.f;
  F2 acc = f2_zero();
  for (int k = blockIdx.x * NT + threadIdx.x; k < nT; k += gridDim.x * NT) {
    const int u = t_unk[k];
    float v = 0.f;
    for (int e = t_ptr[k]; e < t_ptr[k + 1]; ++e) v += t_val[e] * t[t_row[e]];
    const float pu = p[u];
    if (lm) {
      const int c = (int)(u / pl);
      v += lam * dc[cm.mp[c] * pl + (u - c * pl)] * pu;
    }
    q[u] = v;
    f2_add_prod(acc, pu, v);
  }
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, gridDim.x)) {
    double pq, unused;
    gather_partials(part, 0, gridDim.x, &s->counter, pq, unused);
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

// A = J^T J, one thread per row u (a non-empty unknown): for every residual
// row r with an entry J[r,u] (the J^T row of u), every entry J[r,v] of that
// row adds J[r,u] J[r,v] to A[u,v] (v found in u's short sorted column
// list).  The row is owned by one thread, so the sums need no atomics and
// follow a fixed order.
__global__ void __launch_bounds__(NT) k_jtj_assemble(int nT, const int* __restrict__ t_ptr,
                                                     const int* __restrict__ t_row, const float* __restrict__ t_val,
                                                     const int* __restrict__ rp, const int* __restrict__ col,
                                                     const float* __restrict__ val, const int* __restrict__ a_ptr,
                                                     const int* __restrict__ a_col, float* __restrict__ a_val,
                                                     const Scalars* __restrict__ s) {
  if (s->done) return;
  for (int k = blockIdx.x * NT + threadIdx.x; k < nT; k += gridDim.x * NT) {
    const int a0 = a_ptr[k], a1 = a_ptr[k + 1];
    for (int n = a0; n < a1; ++n) a_val[n] = 0.f;
    for (int e = t_ptr[k]; e < t_ptr[k + 1]; ++e) {
      const int r = t_row[e];
      const float ju = t_val[e];
      for (int f = rp[r]; f < rp[r + 1]; ++f) {
        const int v = col[f];
        int lo = a0, hi = a1 - 1;
        while (lo < hi) {                 // the row's columns are sorted
          const int mid = (lo + hi) >> 1;
          if (a_col[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        a_val[lo] += ju * val[f];
      }
    }
  }
}

// q = A p (+ lambda D p) over the non-empty unknowns; float64 p.q -> alpha.
__global__ void __launch_bounds__(NT) k_jtj_spmv(int nT, const int* __restrict__ t_unk, const int* __restrict__ a_ptr,
                                                 const int* __restrict__ a_col, const float* __restrict__ a_val,
                                                 const float* __restrict__ p, float* __restrict__ q,
                                                 const float* __restrict__ dc, int lm, long long pl, CompMap cm,
                                                 Scalars* __restrict__ s, double* __restrict__ part) {
  if (s->done || !s->pcg_active) return;
  const float lam = lm ? s->lambda_f : 0.f;
  F2 acc = f2_zero();
  for (int k = blockIdx.x * NT + threadIdx.x; k < nT; k += gridDim.x * NT) {
    const int u = t_unk[k];
    float v = 0.f;
    for (int n = a_ptr[k]; n < a_ptr[k + 1]; ++n) v += a_val[n] * p[a_col[n]];
    const float pu = p[u];
    if (lm) {
      const int c = (int)(u / pl);
      v += lam * dc[cm.mp[c] * pl + (u - c * pl)] * pu;
    }
    q[u] = v;
    f2_add_prod(acc, pu, v);
  }
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), &s->counter, gridDim.x)) {
    double pq, unused;
    gather_partials(part, 0, gridDim.x, &s->counter, pq, unused);
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

int blocks_for(long long n, int cap) {
  return (int)std::max<long long>(1, std::min<long long>((n + NT - 1) / NT, cap));
}

CompMap comp_map(int kind) {
  CompMap cm{};
  for (int c = 0; c < 6; ++c) cm.mp[c] = kind == K_WARP ? (c == 2 ? 1 : 0) : (kind == K_POISSON ? 0 : (c < 3 ? 0 : c - 2));
  return cm;
}

template <class T>
bool upload_vec(opt_problem* pb, T** dst, const std::vector<T>& v) {
  void* ptr = nullptr;
  const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) return false;
  pb->allocs.push_back(ptr);
  pb->pooled.push_back(false);
  if (!v.empty() && cudaMemcpy(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  *dst = static_cast<T*>(ptr);
  return true;
}

}  // namespace

// Builds the CSR structure of J and J^T (host, once per problem).
static opt_status csr_build_j(opt_problem* pb) {
  CsrJ& J = pb->csr;
  if (J.rp) return OPT_OK;
  const long long pl = pb->plane;
  std::vector<int> rp(1, 0), col;
  std::vector<float> val;
  auto row = [&](std::initializer_list<int> cols, std::initializer_list<float> vals) {
    col.insert(col.end(), cols);
    val.insert(val.end(), vals);
    rp.push_back((int)col.size());
  };
  int groups = 0;
  if (pb->kind == K_WARP || pb->kind == K_POISSON) {
    const int W = pb->W, H = pb->H, P = pb->P;
    const float sw = pb->hg.s_w, sf = pb->hg.s_f;
    auto masked = [&](int x, int y) { return !pb->h_mask.empty() && pb->h_mask[(size_t)y * W + x] != 0; };
    const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        if (masked(x, y)) continue;
        const int i = y * P + x;
        for (int k = 0; k < 4; ++k) {
          const int nx = x + DX[k], ny = y + DY[k];
          if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
          const int j = ny * P + nx;
          if (pb->kind == K_WARP) {
            if (masked(nx, ny)) continue;
            row({i, j, (int)(2 * pl) + i}, {sw, -sw, 0.f});
            row({(int)pl + i, (int)pl + j, (int)(2 * pl) + i}, {sw, -sw, 0.f});
            ++groups;
          } else {
            for (int c = 0; c < 4; ++c) {
              if (masked(nx, ny)) row({(int)(c * pl) + i}, {1.f});
              else row({(int)(c * pl) + i, (int)(c * pl) + j}, {1.f, -1.f});
            }
          }
        }
      }
    if (pb->kind == K_WARP) {
      for (int hp : pb->h_hpix) {
        const int x = hp % P, y = hp / P;
        if (masked(x, y)) continue;
        row({hp}, {sf});
        row({(int)pl + hp}, {sf});
      }
    }
  } else {
    const float sw = pb->hm.s_w, sf = pb->hm.s_f;
    for (size_t e = 0; e < pb->h_e0.size(); ++e) {
      const int a = pb->h_e0[e], b = pb->h_e1[e];
      for (int c = 0; c < 3; ++c)
        row({(int)(c * pl) + a, (int)(c * pl) + b, (int)(3 * pl) + a, (int)(4 * pl) + a, (int)(5 * pl) + a},
            {sw, -sw, 0.f, 0.f, 0.f});
      ++groups;
    }
    for (int h : pb->h_hpix)
      for (int c = 0; c < 3; ++c) row({(int)(c * pl) + h}, {sf});
  }
  const long long nnz = (long long)col.size();
  const int R = (int)rp.size() - 1;
  // transpose by counting sort over the columns
  const long long ncol = (long long)pb->nx * pl;
  std::vector<int> cnt((size_t)ncol + 1, 0);
  for (long long k = 0; k < nnz; ++k) cnt[(size_t)col[k] + 1]++;
  for (long long u = 0; u < ncol; ++u) cnt[(size_t)u + 1] += cnt[(size_t)u];
  std::vector<int> fill(cnt.begin(), cnt.end() - 1), t_row((size_t)nnz), t_perm((size_t)nnz);
  for (int r = 0; r < R; ++r)
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const int pos = fill[(size_t)col[k]]++;
      t_row[pos] = r;
      t_perm[pos] = k;
    }
  std::vector<int> t_unk, t_ptr(1, 0);
  for (long long u = 0; u < ncol; ++u)
    if (cnt[(size_t)u + 1] > cnt[(size_t)u]) {
      t_unk.push_back((int)u);
      t_ptr.push_back(cnt[(size_t)u + 1]);
    }
  J.R = R;
  J.nnz = nnz;
  J.nT = (int)t_unk.size();
  J.ngroups = groups;
  std::vector<float> zeros_R((size_t)R, 0.f), tval((size_t)nnz);
  for (long long k = 0; k < nnz; ++k) tval[k] = val[t_perm[k]];
  if (!upload_vec(pb, &J.rp, rp) || !upload_vec(pb, &J.col, col) || !upload_vec(pb, &J.val, val) ||
      !upload_vec(pb, &J.t_unk, t_unk) || !upload_vec(pb, &J.t_ptr, t_ptr) || !upload_vec(pb, &J.t_row, t_row) ||
      !upload_vec(pb, &J.t_perm, t_perm) || !upload_vec(pb, &J.t_val, tval) || !upload_vec(pb, &J.tvec, zeros_R)) {
    J.rp = nullptr;
    (void)cudaGetLastError();
    return OPT_ERR_OOM;
  }
  J.nblk_t = blocks_for(J.nT, pb->sms * 8);
  std::vector<double> zp((size_t)2 * J.nblk_t, 0.0);
  if (!upload_vec(pb, &J.part, zp)) return OPT_ERR_OOM;
  return OPT_OK;
}

// Pattern of A = J^T J (host, once, for mode 2): the columns of every row that
// shares a residual with unknown t_unk[k], sorted and unique.
static opt_status csr_build_a(opt_problem* pb) {
  CsrJ& J = pb->csr;
  if (J.a_ptr) return OPT_OK;
  std::vector<int> rp((size_t)J.R + 1), col((size_t)J.nnz), t_ptr((size_t)J.nT + 1), t_row((size_t)J.nnz);
  if (cudaMemcpy(rp.data(), J.rp, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(col.data(), J.col, col.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(t_ptr.data(), J.t_ptr, t_ptr.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(t_row.data(), J.t_row, t_row.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    (void)cudaGetLastError();
    return OPT_ERR_CUDA;
  }
  // pattern of A = J^T J: the columns of every row that shares a residual
  // with unknown t_unk[k], sorted and unique
  std::vector<int> a_ptr(1, 0), a_col, scratch;
  a_col.reserve((size_t)J.nT * 16);
  for (int k = 0; k < J.nT; ++k) {
    scratch.clear();
    for (int e = t_ptr[k]; e < t_ptr[(size_t)k + 1]; ++e) {
      const int r = t_row[e];
      for (int f = rp[r]; f < rp[(size_t)r + 1]; ++f) scratch.push_back(col[f]);
    }
    std::sort(scratch.begin(), scratch.end());
    scratch.erase(std::unique(scratch.begin(), scratch.end()), scratch.end());
    a_col.insert(a_col.end(), scratch.begin(), scratch.end());
    a_ptr.push_back((int)a_col.size());
  }
  J.nnz_a = (long long)a_col.size();
  std::vector<float> a_zero(a_col.size(), 0.f);
  if (!upload_vec(pb, &J.a_ptr, a_ptr) || !upload_vec(pb, &J.a_col, a_col) || !upload_vec(pb, &J.a_val, a_zero))
    return OPT_ERR_OOM;
  return OPT_OK;
}

opt_status csr_build(opt_problem* pb, int mode) {
  opt_status st = csr_build_j(pb);
  if (st == OPT_OK && mode == 2) st = csr_build_a(pb);
  return st;
}

// evalJ (once per outer iteration): values that depend on x, then J^T's copy
// and, for the assembled form (mode 2), A = J^T J.
void csr_evalj(opt_problem* pb, cudaStream_t st, int mode) {
  CsrJ& J = pb->csr;
  const int cap = pb->sms * 8;
  if (pb->kind == K_POISSON) {          // constant J (A is still rebuilt once per PCG solve, as in the paper)
    if (mode == 2)
      k_jtj_assemble<<<blocks_for(J.nT, cap), NT, 0, st>>>(J.nT, J.t_ptr, J.t_row, J.t_val, J.rp, J.col, J.val,
                                                           J.a_ptr, J.a_col, J.a_val, pb->d_s);
    return;
  }
  if (pb->kind == K_WARP) {
    k_evalj_warp<<<blocks_for(J.ngroups, cap), NT, 0, st>>>(J.ngroups, J.col, J.val, pb->x, pb->hg.c, pb->plane,
                                                             pb->hg.s_w, pb->d_s);
  } else {
    k_evalj_mesh<<<blocks_for(J.ngroups, cap), NT, 0, st>>>(J.ngroups, pb->hm.e0, pb->hm.e1, J.val, pb->x,
                                                             pb->hm.U, pb->plane, pb->hm.s_w, pb->d_s);
  }
  k_gather_vals<<<blocks_for(J.nnz, cap), NT, 0, st>>>(J.nnz, J.t_perm, J.val, J.t_val, pb->d_s);
  if (mode == 2)
    k_jtj_assemble<<<blocks_for(J.nT, cap), NT, 0, st>>>(J.nT, J.t_ptr, J.t_row, J.t_val, J.rp, J.col, J.val,
                                                         J.a_ptr, J.a_col, J.a_val, pb->d_s);
}

// One materialized applyJTJ: direction update, then t = J p, q = J^T t
// (mode 1) or q = A p (mode 2), plus damping.
void csr_apply(opt_problem* pb, cudaStream_t st, int par, int mode) {
  CsrJ& J = pb->csr;
  const int cap = pb->sms * 8;
  const CompMap cm = comp_map(pb->kind);
  const long long pl = pb->plane;
  const float* pin = pb->pbuf + (long long)(par & 1) * pb->nx * pl;
  float* pout = pb->pbuf + (long long)((par + 1) & 1) * pb->nx * pl;
  const bool graph = pb->kind == K_MESH || pb->kind == K_VOLUME;   // the mesh energy (K_WARPG has no CSR form)
  const float* m = graph ? pb->hm.m : pb->hg.m;
  const float* dc = graph ? pb->hm.dc : pb->hg.dc;
  const int lm = graph ? pb->hm.lm : pb->hg.lm;
  k_csr_direction<<<blocks_for(J.nT, cap), NT, 0, st>>>(J.nT, J.t_unk, pl, cm, m, pb->rvec, pin, pout, pb->d_s);
  if (mode == 2) {
    k_jtj_spmv<<<J.nblk_t, NT, 0, st>>>(J.nT, J.t_unk, J.a_ptr, J.a_col, J.a_val, pout, pb->qvec, dc, lm, pl, cm,
                                        pb->d_s, J.part);
    return;
  }
  k_csr_jp<<<blocks_for(J.R, cap), NT, 0, st>>>(J.R, J.rp, J.col, J.val, pout, J.tvec, pb->d_s);
  k_csr_jtt<<<J.nblk_t, NT, 0, st>>>(J.nT, J.t_unk, J.t_ptr, J.t_row, J.t_val, J.tvec, pout, pb->qvec, dc, lm, pl,
                                     cm, pb->d_s, J.part);
}

}  // namespace optgb
