// Allocation-free variant of the fused step kernel (cavity_step_block_noalloc
// in include/cavity.h).
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or a pre-sized arena, where allocating from the
// driver behind that allocator's back would break its accounting or its
// out-of-memory handling.  This entry point lets such a caller run one fused
// residual + update pass over one block it already holds in device memory:
// the caller passes the input state, the output state and a 6-double output,
// and the reduction scratch the kernel needs lives in a fixed array compiled
// into the library (g_noalloc_scratch below), so no call allocates anything.
//
// The array exists once per GPU that loads the library and stays allocated
// until the process exits.  Every call shares it and it keeps the previous
// call's contents; each call overwrites all of it that it reads (descriptors
// and one partial slot per CTA), so nothing needs clearing.  Two calls whose
// work overlaps on a GPU (on different streams, or from different threads)
// race on the array and give wrong results.
//
// The paper has no counterpart: it describes no memory-management constraint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/cavity.h"
#include "bdc_device.cuh"

using namespace bdc;

namespace {

constexpr int kTX = 32, kTY = 8, kKC = 16;  // the tile of the FP64 step kernel
constexpr int kDescBytes = 1280;           // BlockDev (256) + CavConst (768) + CavState (256), aligned slots
constexpr size_t kScratchBytes = kDescBytes + (size_t)CAVITY_NOALLOC_MAX_TILES * kPartStride * sizeof(double);
constexpr int kMaxDevices = 64;

static_assert(sizeof(BlockDev) <= 256 && sizeof(CavConst) <= 768 && sizeof(CavState) <= 256,
              "descriptor slots too small");

// reduction scratch and descriptors of the allocation-free entry point
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side name of the array is not a device address).
cudaError_t scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Writes the three descriptors into the scratch array.  They arrive as kernel
// parameters, which the launch copies by value, so the call reads no host
// memory after it returns and makes no host-to-device copy of its own.
__global__ void k_noalloc_setup(BlockDev B, CavConst C, CavState S, BlockDev *d_block, CavConst *d_cc,
                                CavState *d_cs) {
  if (threadIdx.x == 0) {
    *d_block = B;
    *d_cc = C;
    *d_cs = S;
  }
}

// RMS of the five rates and the next dt from the per-CTA partials, summed in
// a fixed order (thread q takes partials q, q + 256, ...; warps in order)
__global__ void __launch_bounds__(256) k_noalloc_reduce(const double *partials, int ntiles, const CavConst *cc,
                                                        double *out6) {
  __shared__ double sh[8][6];
  const int tid = threadIdx.x;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int q = tid; q < ntiles; q += 256) {
    const double *pp = partials + (long long)q * kPartStride;
    for (int f = 0; f < 5; ++f) acc[f] += pp[f];
    acc[5] = fmax(acc[5], pp[5]);
  }
  for (int f = 0; f < 5; ++f) acc[f] = warp_sum(acc[f]);
  acc[5] = warp_max(acc[5]);
  if ((tid & 31) == 0)
    for (int f = 0; f < 6; ++f) sh[tid >> 5][f] = acc[f];
  __syncthreads();
  if (tid == 0) {
    double tot[6];
    for (int f = 0; f < 6; ++f) tot[f] = sh[0][f];
    for (int w = 1; w < 8; ++w)
      for (int f = 0; f < 6; ++f) tot[f] = (f == 5) ? fmax(tot[f], sh[w][f]) : tot[f] + sh[w][f];
    for (int f = 0; f < 5; ++f) out6[f] = sqrt(tot[f] * cc->inv_nint);
    out6[5] = cc->cfl / tot[5];
  }
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

extern "C" CAVITY_API int cavity_step_block_noalloc(const double *q_in, double *q_out, int nx, int ny, int nz,
                                                    const cavity_params *p, double dt, double pshift,
                                                    double *out6, void *stream) {
  if (!q_in || !q_out || !out6 || !p || q_in == q_out) return CAVITY_ERR_INVALID_ARG;
  if (nx < 2 || ny < 2 || nz < 2 || !(dt >= 0.0) || !std::isfinite(pshift)) return CAVITY_ERR_INVALID_ARG;
  const long long ntiles = (long long)ceil_div(nx, kTX) * ceil_div(ny, kTY) * ceil_div(nz, kKC);
  if (ntiles > CAVITY_NOALLOC_MAX_TILES) return CAVITY_ERR_INVALID_ARG;  // beyond the fixed scratch
  cavity_params q = *p;
  if (!(q.u_ref >= 0.0)) q.u_ref = std::max(1.0, std::sqrt(q.Ra * q.Pr));
  if (std::isnan(q.t_inf)) q.t_inf = 0.5 * (q.t_hot + q.t_cold);
  if (!(q.Ra >= 0.0) || !(q.Pr > 0.0) || !(q.cfl > 0.0) || !(q.kappa > 0.0) || !(q.c4 >= 0.0) ||
      !(q.u_ref > 0.0) || !std::isfinite(q.t_inf) || (q.gravity_axis != 1 && q.gravity_axis != 2))
    return CAVITY_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CAVITY_ERR_CUDA;
  void *scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return CAVITY_ERR_CUDA;
  unsigned char *s = (unsigned char *)scratch;
  BlockDev *d_block = (BlockDev *)s;
  CavConst *d_cc = (CavConst *)(s + 256);
  CavState *d_cs = (CavState *)(s + 1024);
  double *d_part = (double *)(s + kDescBytes);

  // dense caller layout: node (i, j, k), i in [-1, n+2], at (i+1) + (nx+4)((j+1) + (ny+4)(k+1));
  // the kernel addresses node i at XO - 1 + i, so the base is moved back by XO - 2 elements
  BlockDev B{};
  B.nx = nx; B.ny = ny; B.nz = nz;
  B.pitch = nx + 4;
  B.rows = ny + 4;
  B.plane = (long long)B.pitch * B.rows;
  B.fstride = B.plane * (nz + 4);
  for (int f = 0; f < 6; ++f) { B.wall[f] = 1; B.nbr[f] = -1; }
  B.tiles_x = ceil_div(nx, kTX);
  B.tiles_y = ceil_div(ny, kTY);
  B.tiles_z = ceil_div(nz, kKC);
  B.tiles_zc = B.tiles_z;  // one CTA per tile: KC-plane chunks only
  B.zsplit = nz;
  B.coarse_begin = 0;
  B.fine_begin = 0;
  B.base[0] = (void *)(q_in - (XO<double>::v - 2));
  B.base[1] = (void *)(q_out - (XO<double>::v - 2));

  CavConst C{};
  const int gn[3] = {nx, ny, nz};
  set_cav_physics(C, gn, q);

  CavState S{};
  S.dt = dt;
  S.c = pshift;

  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_setup<<<1, 32, 0, st>>>(B, C, S, d_block, d_cc, d_cs);
  if (cudaGetLastError() != cudaSuccess) return CAVITY_ERR_CUDA;
  StepArgs a{};  // tile_counter null: one CTA per tile
  a.blocks = d_block; a.nblocks = 1; a.cc = d_cc; a.cs = d_cs;
  a.partials = d_part; a.parity = 0; a.mode = 0; a.ntiles = (int)ntiles;
  a.ncoarse = (int)ntiles;
  k_step_f64<kTX, kTY, kKC><<<(int)ntiles, dim3(kTX, kTY), 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return CAVITY_ERR_CUDA;
  k_noalloc_reduce<<<1, 256, 0, st>>>(d_part, (int)ntiles, d_cc, out6);
  if (cudaGetLastError() != cudaSuccess) return CAVITY_ERR_CUDA;
  return CAVITY_OK;
}
