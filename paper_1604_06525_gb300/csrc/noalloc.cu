// Allocation-free J^T J p for the ARAP image warp.
//
// Some callers cannot call cudaMalloc: interactive editing loops that run on
// a fixed per-frame time budget and must not stall on an allocation (or on the
// device-wide synchronisation cudaMalloc / cudaFree may imply), and host
// applications or plug-in hosts that own all device memory through their own
// allocator and hand a component only the buffers it works on.  For them this
// file provides opt_warp_apply_jtj_noalloc: the same product as
// opt_apply_jtj on an ARAP warp (lambda = 0), reading the caller's dense planes
// directly, with its only scratch -- the float64 per-block partial sums of
// p.q and the arrival counter of the last-block reduction -- in the
// file-scope array below.  It calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array lives on every device that loads this library until the process
// exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; that
// first call should therefore come before any stream capture.  Every call
// shares the array (the counter is cleared at the start of each call, the
// partial slots are always written before they are read); calls whose
// kernels overlap on the GPU race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "opt_gb300.h"
#include "opt_internal.cuh"

using namespace optgb;

namespace {

// 256-byte header (arrival counter) + two float64 partial slots per 32x8
// tile: 256 B + 16 * OPT_NOALLOC_MAX_TILES B = 262,400 bytes per device.
constexpr int kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + 2 * sizeof(double) * OPT_NOALLOC_MAX_TILES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ int na_dx(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
__device__ __forceinline__ int na_dy(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }

// One block per 32x8 tile, dense planes (row pitch W).  Same algebra as the
// matrix-free warp product: own residual rows s_w[(p_i - p_j) - R'(t_i) v p_t,i],
// incoming rows s_w[(p_j - p_i) - R'(t_j)(-v) p_t,j], fit rows w_fit p_i.
__global__ void __launch_bounds__(NT) k_warp_apply_noalloc(
    int W, int H, const float* __restrict__ x, const float* __restrict__ U,
    const uint8_t* __restrict__ mask, const int* __restrict__ hidx, int nh, float sw, float wfit,
    const float* __restrict__ p, float* __restrict__ q, double* __restrict__ pq_out,
    unsigned char* __restrict__ scratch) {
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
  double* part = reinterpret_cast<double*>(scratch + kHeaderBytes);
  __shared__ float sp[3][HH][HW], scs[HH][HW], ssn[HH][HW], sux[HH][HW], suy[HH][HW];
  __shared__ unsigned char sv[HH][HW];
  __shared__ int sfit[TH][TW];      // handle entries on each pixel of the tile
  const long long pl = (long long)W * H;
  const int ntx = (W + TW - 1) / TW;
  const int x0 = (blockIdx.x % ntx) * TW, y0 = (blockIdx.x / ntx) * TH;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  sfit[ty][tx] = 0;
  for (int hc = threadIdx.x; hc < HW * HH; hc += NT) {
    const int hy = hc / HW, hx = hc - hy * HW;
    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
    float a = 0.f, b = 0.f, c = 0.f, th = 0.f, ux = 0.f, uy = 0.f;
    unsigned char v = 0;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const long long i = (long long)gy * W + gx;
      a = p[i]; b = p[pl + i]; c = p[2 * pl + i];
      th = x[2 * pl + i];
      ux = U[i]; uy = U[pl + i];
      v = mask ? (mask[i] == 0) : 1;
    }
    float sn, cs;
    sincosf(th, &sn, &cs);
    sp[0][hy][hx] = a; sp[1][hy][hx] = b; sp[2][hy][hx] = c;
    scs[hy][hx] = cs; ssn[hy][hx] = sn; sux[hy][hx] = ux; suy[hy][hx] = uy; sv[hy][hx] = v;
  }
  __syncthreads();
  // every block scans the whole handle list (O(tiles x n_handles) loads);
  // a repeated index counts once per entry, as a sum of squares over entries
  for (int h = threadIdx.x; h < nh; h += NT) {
    const int pix = hidx[h];
    const int hx = pix % W - x0, hy = pix / W - y0;
    if (hx >= 0 && hx < TW && hy >= 0 && hy < TH) atomicAdd(&sfit[hy][hx], 1);
  }
  __syncthreads();
  F2 acc = f2_zero();
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < W && gy < H) {
    const int lx = tx + 1, ly = ty + 1;
    const long long i = (long long)gy * W + gx;
    const float pxi = sp[0][ly][lx], pyi = sp[1][ly][lx], pti = sp[2][ly][lx];
    float qx = 0.f, qy = 0.f, qt = 0.f;
    if (sv[ly][lx]) {
      const float ci = scs[ly][lx], si = ssn[ly][lx];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nx = lx + na_dx(k), ny = ly + na_dy(k);
        if (!sv[ny][nx]) continue;
        const float vx = sux[ly][lx] - sux[ny][nx], vy = suy[ly][lx] - suy[ny][nx];
        const float pxj = sp[0][ny][nx], pyj = sp[1][ny][nx], ptj = sp[2][ny][nx];
        const float gx_ = -sw * (-si * vx - ci * vy), gy_ = -sw * (ci * vx - si * vy);
        const float jpx = sw * (pxi - pxj) + gx_ * pti, jpy = sw * (pyi - pyj) + gy_ * pti;
        qx += sw * jpx;
        qy += sw * jpy;
        qt += gx_ * jpx + gy_ * jpy;
        const float cj = scs[ny][nx], sj = ssn[ny][nx];
        const float hx_ = -sw * (sj * vx + cj * vy), hy_ = -sw * (-cj * vx + sj * vy);
        qx -= sw * (sw * (pxj - pxi) + hx_ * ptj);
        qy -= sw * (sw * (pyj - pyi) + hy_ * ptj);
      }
      if (sfit[ty][tx]) {
        const float wf = wfit * (float)sfit[ty][tx];
        qx += wf * pxi;
        qy += wf * pyi;
      }
    }
    q[i] = qx; q[pl + i] = qy; q[2 * pl + i] = qt;
    f2_add_prod(acc, pxi, qx);
    f2_add_prod(acc, pyi, qy);
    f2_add_prod(acc, pti, qt);
  }
  if (publish_partials(part, blockIdx.x, acc, f2_zero(), counter, gridDim.x)) {
    double pq, unused;
    gather_partials(part, 0, gridDim.x, counter, pq, unused);
    if (threadIdx.x == 0 && pq_out) *pq_out = pq;
  }
}

// Device address of the scratch array for the current device (looked up on
// the first call for that device).
opt_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OPT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      (void)cudaGetLastError();
      return OPT_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return OPT_OK;
}

}  // namespace

extern "C" opt_status opt_warp_apply_jtj_noalloc(int32_t W, int32_t H, const float* x, const float* urshape,
                                                 const uint8_t* mask, const int32_t* handle_idx,
                                                 int32_t n_handles, float w_reg, float w_fit,
                                                 const float* p, float* q, double* pq, void* stream) {
  if (W < 1 || H < 1 || W >= 32768 || H >= 32768) return OPT_ERR_INVALID_ARG;
  const long long tiles = (long long)((W + TW - 1) / TW) * ((H + TH - 1) / TH);
  if (tiles > OPT_NOALLOC_MAX_TILES) return OPT_ERR_INVALID_ARG;
  if (!x || !urshape || !p || !q || n_handles < 0 || (n_handles > 0 && !handle_idx)) return OPT_ERR_INVALID_ARG;
  if (!(w_reg >= 0.f) || !(w_fit >= 0.f)) return OPT_ERR_INVALID_ARG;
  void* scratch = nullptr;
  const opt_status s = scratch_for_current_device(&scratch);
  if (s != OPT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(scratch, 0, kHeaderBytes, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return OPT_ERR_CUDA;
  }
  k_warp_apply_noalloc<<<(unsigned)tiles, NT, 0, st>>>(W, H, x, urshape, mask, handle_idx, n_handles,
                                                       sqrtf(w_reg), w_fit, p, q, pq,
                                                       static_cast<unsigned char*>(scratch));
  if (cudaGetLastError() != cudaSuccess) return OPT_ERR_CUDA;
  return OPT_OK;
}
