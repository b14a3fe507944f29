// C ABI of the buoyancy-driven-cavity step (include/cavity.h): host runtime
// that lays out the blocks in HBM, builds the work lists of the kernels in
// bdc_device.cuh / bdc_step_f32.cuh, captures one CUDA graph per buffer
// parity and replays it.  Two arithmetic forms share the runtime: FP64
// (five FP64 arrays per buffer set) and FP32-mixed (p_hi, p_lo, u, v, w, T in
// FP32, read by the step kernel through TMA tensor maps).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cavity.h"
#include "bdc_device.cuh"
#include "bdc_step_f32.cuh"

using namespace bdc;

namespace {

constexpr int kTX = 32, kTY = 8, kKC = 16;  // k_step tile of the FP64 form

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

std::vector<int> split_sizes(int n, int parts) {  // Section 3.2: as even as possible
  std::vector<int> s(parts, n / parts);
  for (int r = 0; r < n % parts; ++r) s[r] += 1;
  return s;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

struct cavity {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cavity_desc desc{};
  cavity_params prm{};
  bool f32 = false;  // FP32-mixed form
  size_t esize = 8;  // bytes per stored element
  int na = 5;        // stored arrays per buffer set
  int np = 1;        // pressure arrays
  int tx = kTX, ty = kTY, kc = kKC;
  int f32_r = 0;  // ring depth of the FP32 step kernel
  int nblocks = 0;
  std::vector<BlockDev> hb;
  std::vector<WallFace> hwall;
  std::vector<WallFace> hnus;  // x-wall faces (Nusselt-only wall pass)
  std::vector<CutFace> hcut;
  CavConst hcc{};
  long long xbuf_elems = 0;
  int n_step = 0, n_bc = 0, n_cut = 0, n_nus = 0;
  WallFace *d_nus = nullptr;

  BlockDev *d_blocks = nullptr;
  CavConst *d_cc = nullptr;
  CavState *d_cs = nullptr;
  WallFace *d_wall = nullptr;
  CutFace *d_cut = nullptr;
  CUtensorMap *d_maps = nullptr;
  double *d_step_part = nullptr, *d_bc_part = nullptr, *d_twall = nullptr, *d_stage = nullptr;
  unsigned int *d_counter = nullptr;
  void *d_fields = nullptr, *d_xbuf = nullptr;
  size_t field_bytes = 0;
  size_t stage_elems = 0;

  std::vector<double> twall;  // hot wall then cold wall, gny*gnz each
  bool wall_custom[2] = {false, false};
  int parity = 0;
  long long steps_taken = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::string err;
};

namespace {

int fail(cavity *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(h, e_ == cudaErrorMemoryAllocation ? CAVITY_ERR_OOM : CAVITY_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int xo1(size_t esize) { return esize == 8 ? XO<double>::v : XO<float>::v; }

long long host_node_index(const BlockDev &B, size_t esize, int i, int j, int k) {
  return (long long)(xo1(esize) - 1 + i) + (long long)B.pitch * (j + 1) + B.plane * (k + 1);
}

void fill_consts(cavity *h) {
  CavConst &C = h->hcc;
  const cavity_params &p = h->prm;
  const int gn[3] = {h->desc.nx, h->desc.ny, h->desc.nz};
  double sih = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double np1 = (double)gn[d] + 1.0;
    C.gn[d] = gn[d];
    C.h[d] = 1.0 / np1;
    C.ih[d] = np1;
    C.ih2[d] = 0.5 * np1;
    C.ihh[d] = np1 * np1;
    sih += C.ihh[d];
  }
  C.nu = p.Pr;
  C.alpha = 1.0;
  C.gs = p.Ra * p.Pr;
  C.t_inf = p.t_inf;
  C.b2min = p.kappa * p.u_ref * p.u_ref;
  C.c4 = p.c4;
  C.cfl = p.cfl;
  C.diffsr = 2.0 * std::max(C.nu, C.alpha) * sih;
  C.inv_dT = 1.0 / (p.t_hot - p.t_cold);
  C.inv_nint = 1.0 / ((double)gn[0] * gn[1] * gn[2]);
  C.inv_nwall = 1.0 / ((double)gn[1] * gn[2]);
  C.gaxis = p.gravity_axis;
}

void resolve_defaults(cavity_params *p) {
  if (!(p->u_ref >= 0.0)) p->u_ref = std::max(1.0, std::sqrt(p->Ra * p->Pr));
  if (std::isnan(p->t_inf)) p->t_inf = 0.5 * (p->t_hot + p->t_cold);
}

int check_params(const cavity_params &p) {
  if (!(p.Ra >= 0.0) || !(p.Pr > 0.0) || !(p.cfl > 0.0) || !(p.kappa > 0.0) || !(p.c4 >= 0.0) ||
      !(p.u_ref > 0.0) || !std::isfinite(p.t_inf) || !std::isfinite(p.t_hot) || !std::isfinite(p.t_cold) ||
      p.t_hot == p.t_cold || (p.gravity_axis != 1 && p.gravity_axis != 2))
    return CAVITY_ERR_INVALID_ARG;
  return CAVITY_OK;
}

// ---------------------------------------------------------------------------
int build_layout(cavity *h) {
  const cavity_desc &d = h->desc;
  const int gn[3] = {d.nx, d.ny, d.nz};
  const int pg[3] = {d.px, d.py, d.pz};
  std::vector<int> sz[3], org[3];
  for (int a = 0; a < 3; ++a) {
    sz[a] = split_sizes(gn[a], pg[a]);
    int o = 0;
    for (int s : sz[a]) { org[a].push_back(o); o += s; }
  }
  const size_t es = h->esize;
  const int row_align = (int)(128 / es);
  h->nblocks = pg[0] * pg[1] * pg[2];
  h->hb.assign(h->nblocks, BlockDev{});
  size_t total_elems = 0;
  int tile = 0;
  for (int bz = 0; bz < pg[2]; ++bz)
    for (int by = 0; by < pg[1]; ++by)
      for (int bx = 0; bx < pg[0]; ++bx) {
        const int id = bx + pg[0] * (by + pg[1] * bz);
        BlockDev &B = h->hb[id];
        B.nx = sz[0][bx]; B.ny = sz[1][by]; B.nz = sz[2][bz];
        B.ox = org[0][bx]; B.oy = org[1][by]; B.oz = org[2][bz];
        B.pitch = ((xo1(es) + B.nx + 2 + row_align - 1) / row_align) * row_align;
        B.rows = B.ny + 4;
        B.plane = (long long)B.pitch * B.rows;
        B.fstride = ((B.plane * (B.nz + 4) + 63) / 64) * 64;
        const int c[3] = {bx, by, bz};
        for (int f = 0; f < 6; ++f) {
          const int a = f / 2, hi = f % 2;
          int cc[3] = {c[0], c[1], c[2]};
          cc[a] += hi ? 1 : -1;
          const bool inside = cc[a] >= 0 && cc[a] < pg[a];
          B.wall[f] = inside ? 0 : 1;
          B.nbr[f] = inside ? cc[0] + pg[0] * (cc[1] + pg[1] * cc[2]) : -1;
        }
        B.cav = 0;
        B.tiles_x = ceil_div(B.nx, h->tx);
        B.tiles_y = ceil_div(B.ny, h->ty);
        B.tiles_z = ceil_div(B.nz, h->kc);
        B.tile_begin = tile;
        tile += B.tiles_x * B.tiles_y * B.tiles_z;
        total_elems += 2 * (size_t)h->na * (size_t)B.fstride;
      }
  h->n_step = tile;
  h->field_bytes = total_elems * es;
  // wall and cut faces
  int bc = 0, cut = 0;
  long long xoff = 0;
  h->hwall.clear();
  h->hcut.clear();
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    const int n[3] = {B.nx, B.ny, B.nz};
    for (int f = 0; f < 6; ++f) {
      const int a = f / 2;
      const int n1 = n[a == 0 ? 1 : 0], n2 = n[a == 2 ? 1 : 2];
      if (B.wall[f]) {
        WallFace w{id, f, n1, n2, bc, 0};
        h->hwall.push_back(w);
        bc += ceil_div((long long)n1 * n2, kBcThreads);
      } else {
        CutFace c{id, f, B.nbr[f], n1, n2, cut, xoff};
        h->hcut.push_back(c);
        cut += ceil_div((long long)n1 * n2, 256);
        xoff += (long long)(2 * h->np + 4) * n1 * n2;
      }
    }
  }
  h->n_bc = bc;
  h->n_cut = cut;
  h->xbuf_elems = xoff;
  int nus = 0;
  h->hnus.clear();
  for (const WallFace &w : h->hwall) {
    if (w.face / 2 != 0) continue;
    WallFace x = w;
    x.cta_begin = nus;
    h->hnus.push_back(x);
    nus += ceil_div((long long)w.n1 * w.n2, kBcThreads);
  }
  h->n_nus = nus;
  // cavity constants: work ranges and centre nodes
  CavConst &C = h->hcc;
  C.tile_begin = 0; C.tile_end = h->n_step;
  C.bc_begin = 0; C.bc_end = h->n_bc;
  C.nus_begin = 0; C.nus_end = h->n_nus;
  C.wall_off = 0;
  std::vector<int> ax[3];
  for (int a = 0; a < 3; ++a) {
    if (gn[a] % 2 == 1) ax[a] = {(gn[a] + 1) / 2};
    else ax[a] = {gn[a] / 2, gn[a] / 2 + 1};
  }
  int m = 0;
  for (int K : ax[2])
    for (int J : ax[1])
      for (int I : ax[0]) {
        for (int id = 0; id < h->nblocks; ++id) {
          const BlockDev &B = h->hb[id];
          if (I > B.ox && I <= B.ox + B.nx && J > B.oy && J <= B.oy + B.ny && K > B.oz && K <= B.oz + B.nz) {
            C.centre_blk[m] = id;
            C.centre_off[m] = host_node_index(B, es, I - B.ox, J - B.oy, K - B.oz);
          }
        }
        ++m;
      }
  C.ncentre = m;
  return CAVITY_OK;
}

// FP32 step-kernel variants compiled in: (z chunk KC, ring depth R)
#define BDC_F32_VARIANTS(X) X(16, 8) X(32, 8) X(64, 4) X(64, 8)

bool f32_variant_ok(int kc, int r) {
#define BDC_OK(KC, R) if (kc == KC && r == R) return true;
  BDC_F32_VARIANTS(BDC_OK)
#undef BDC_OK
  return false;
}

cudaError_t f32_set_smem(int kc, int r) {
#define BDC_ATTR(KC, R)                                                                                   \
  if (kc == KC && r == R)                                                                                 \
    return cudaFuncSetAttribute(k_step_f32<KC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                f32_smem_bytes(R));
  BDC_F32_VARIANTS(BDC_ATTR)
#undef BDC_ATTR
  return cudaErrorInvalidValue;
}

// TMA descriptors of the FP32-mixed step kernel: one 4-D map per block and
// buffer set over (x, y, z, array), box = one tile plane with its halo for
// all six arrays
int encode_maps(cavity *h) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) return fail(h, CAVITY_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  EncodeTiledFn encode = (EncodeTiledFn)fn;
  std::vector<CUtensorMap> maps(2 * h->nblocks);
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    for (int s = 0; s < 2; ++s) {
      const cuuint64_t dims[4] = {(cuuint64_t)B.pitch, (cuuint64_t)B.rows, (cuuint64_t)(B.nz + 4), (cuuint64_t)kF32NA};
      const cuuint64_t strides[3] = {(cuuint64_t)B.pitch * 4, (cuuint64_t)B.plane * 4, (cuuint64_t)B.fstride * 4};
      const cuuint32_t box[4] = {(cuuint32_t)kF32BX, (cuuint32_t)kF32BY, 1, (cuuint32_t)kF32NA};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      const CUresult r = encode(&maps[2 * id + s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, B.base[s], dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(h, CAVITY_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
  }
  CK(cudaMalloc(&h->d_maps, sizeof(CUtensorMap) * maps.size()));
  CK(cudaMemcpy(h->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
  return CAVITY_OK;
}

int alloc_device(cavity *h) {
  CK(cudaMalloc(&h->d_fields, h->field_bytes));
  CK(cudaMemsetAsync(h->d_fields, 0, h->field_bytes, h->stream));
  char *base = (char *)h->d_fields;
  for (auto &B : h->hb) {
    for (int s = 0; s < 2; ++s) {
      B.base[s] = base;
      base += (size_t)h->na * (size_t)B.fstride * h->esize;
    }
  }
  CK(cudaMalloc(&h->d_blocks, sizeof(BlockDev) * h->nblocks));
  CK(cudaMalloc(&h->d_cc, sizeof(CavConst)));
  CK(cudaMalloc(&h->d_cs, sizeof(CavState)));
  CK(cudaMemsetAsync(h->d_cs, 0, sizeof(CavState), h->stream));
  CK(cudaMalloc(&h->d_wall, sizeof(WallFace) * std::max<size_t>(1, h->hwall.size())));
  CK(cudaMalloc(&h->d_cut, sizeof(CutFace) * std::max<size_t>(1, h->hcut.size())));
  CK(cudaMalloc(&h->d_nus, sizeof(WallFace) * std::max<size_t>(1, h->hnus.size())));
  if (!h->hnus.empty())
    CK(cudaMemcpyAsync(h->d_nus, h->hnus.data(), sizeof(WallFace) * h->hnus.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMalloc(&h->d_step_part, sizeof(double) * kPartStride * std::max(1, h->n_step)));
  CK(cudaMalloc(&h->d_bc_part, sizeof(double) * 2 * std::max(1, h->n_bc)));
  CK(cudaMalloc(&h->d_counter, sizeof(unsigned int)));
  CK(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned int), h->stream));
  CK(cudaMalloc(&h->d_twall, sizeof(double) * 2 * (size_t)h->desc.ny * h->desc.nz));
  if (h->xbuf_elems > 0) CK(cudaMalloc(&h->d_xbuf, h->esize * (size_t)h->xbuf_elems));
  CK(cudaMemcpyAsync(h->d_blocks, h->hb.data(), sizeof(BlockDev) * h->nblocks, cudaMemcpyHostToDevice, h->stream));
  if (!h->hwall.empty())
    CK(cudaMemcpyAsync(h->d_wall, h->hwall.data(), sizeof(WallFace) * h->hwall.size(), cudaMemcpyHostToDevice, h->stream));
  if (!h->hcut.empty())
    CK(cudaMemcpyAsync(h->d_cut, h->hcut.data(), sizeof(CutFace) * h->hcut.size(), cudaMemcpyHostToDevice, h->stream));
  if (h->f32) {
    int rc = encode_maps(h);
    if (rc != CAVITY_OK) return rc;
    CK(f32_set_smem(h->kc, h->f32_r));
  }
  return CAVITY_OK;
}

int upload_consts(cavity *h) {
  fill_consts(h);
  const size_t nw = (size_t)h->desc.ny * h->desc.nz;
  if (h->twall.size() != 2 * nw) h->twall.assign(2 * nw, 0.0);
  if (!h->wall_custom[0]) std::fill(h->twall.begin(), h->twall.begin() + nw, h->prm.t_hot);
  if (!h->wall_custom[1]) std::fill(h->twall.begin() + nw, h->twall.end(), h->prm.t_cold);
  CK(cudaMemcpyAsync(h->d_cc, &h->hcc, sizeof(CavConst), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_twall, h->twall.data(), sizeof(double) * h->twall.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));  // the host vectors may change after return
  return CAVITY_OK;
}

// ---------------------------------------------------------------------------
// kernel launches

StepArgs step_args(cavity *h, int parity, int mode) {
  StepArgs a;
  a.blocks = h->d_blocks; a.nblocks = h->nblocks; a.cc = h->d_cc; a.cs = h->d_cs;
  a.partials = h->d_step_part; a.parity = parity; a.mode = mode;
  return a;
}

StepF32Args step_f32_args(cavity *h, int parity) {
  StepF32Args a;
  a.blocks = h->d_blocks; a.nblocks = h->nblocks; a.cc = h->d_cc; a.cs = h->d_cs;
  a.maps = h->d_maps; a.partials = h->d_step_part; a.parity = parity;
  return a;
}

BcArgs bc_args(cavity *h, int parity, int mode) {
  BcArgs a;
  a.blocks = h->d_blocks;
  a.faces = mode == 2 ? h->d_nus : h->d_wall;
  a.nfaces = (int)(mode == 2 ? h->hnus.size() : h->hwall.size());
  a.cc = h->d_cc; a.cs = h->d_cs; a.ncav = 1;
  a.step_partials = h->d_step_part; a.bc_partials = h->d_bc_part; a.counter = h->d_counter;
  a.t_wall = h->d_twall; a.parity = parity; a.mode = mode;
  return a;
}

ExchArgs exch_args(cavity *h, int parity) {
  ExchArgs a;
  a.blocks = h->d_blocks; a.faces = h->d_cut; a.nfaces = (int)h->hcut.size();
  a.buf = (double *)h->d_xbuf; a.parity = parity;
  return a;
}

void launch_step_kernel(cavity *h, int parity) {
  if (h->f32) {
#define BDC_LAUNCH(KC, R)                                                                                   \
  if (h->kc == KC && h->f32_r == R)                                                                         \
    k_step_f32<KC, R><<<h->n_step, dim3(kF32TX, kF32TY), f32_smem_bytes(R), h->stream>>>( \
        step_f32_args(h, parity));
    BDC_F32_VARIANTS(BDC_LAUNCH)
#undef BDC_LAUNCH
  } else {
    k_step_f64<kTX, kTY, kKC><<<h->n_step, dim3(kTX, kTY), 0, h->stream>>>(step_args(h, parity, 0));
  }
}

// mode 0: after a step; mode 1: state refresh.  The FP32 step kernel applies
// the walls itself, so after its steps only the Nusselt sums remain (mode 2).
void launch_bc_kernel(cavity *h, int parity, int mode) {
  if (h->f32) {
    if (mode == 0) k_bc<float><<<h->n_nus, kBcThreads, 0, h->stream>>>(bc_args(h, parity, 2));
    else k_bc<float><<<h->n_bc, kBcThreads, 0, h->stream>>>(bc_args(h, parity, mode));
  } else {
    k_bc<double><<<h->n_bc, kBcThreads, 0, h->stream>>>(bc_args(h, parity, mode));
  }
}

void launch_pack(cavity *h, int parity) {
  if (h->f32) k_pack<float><<<h->n_cut, 256, 0, h->stream>>>(exch_args(h, parity));
  else k_pack<double><<<h->n_cut, 256, 0, h->stream>>>(exch_args(h, parity));
}

void launch_unpack(cavity *h, int parity) {
  if (h->f32) k_unpack<float><<<h->n_cut, 256, 0, h->stream>>>(exch_args(h, parity));
  else k_unpack<double><<<h->n_cut, 256, 0, h->stream>>>(exch_args(h, parity));
}

int launch_exchange(cavity *h, int parity) {
  if (h->n_cut == 0) return CAVITY_OK;
  launch_pack(h, parity);
  CK(cudaGetLastError());
  launch_unpack(h, parity);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// one explicit step reading buffer set `parity`, leaving the new state in parity ^ 1
int launch_step(cavity *h, int parity) {
  launch_step_kernel(h, parity);
  CK(cudaGetLastError());
  launch_bc_kernel(h, parity ^ 1, 0);
  CK(cudaGetLastError());
  return launch_exchange(h, parity ^ 1);
}

// walls, ghosts, dt and Nusselt of the state in the current buffer set (no step)
int refresh_state(cavity *h) {
  if (h->f32) {
    const StepArgs sa = step_args(h, h->parity, 1);
    if (h->kc == 16) k_spectral<float, kF32TX, kF32TY, 16><<<h->n_step, dim3(kF32TX, kF32TY), 0, h->stream>>>(sa);
    else if (h->kc == 32) k_spectral<float, kF32TX, kF32TY, 32><<<h->n_step, dim3(kF32TX, kF32TY), 0, h->stream>>>(sa);
    else k_spectral<float, kF32TX, kF32TY, 64><<<h->n_step, dim3(kF32TX, kF32TY), 0, h->stream>>>(sa);
  } else
    k_step_f64<kTX, kTY, kKC><<<h->n_step, dim3(kTX, kTY), 0, h->stream>>>(step_args(h, h->parity, 1));
  CK(cudaGetLastError());
  launch_bc_kernel(h, h->parity, 1);
  CK(cudaGetLastError());
  return launch_exchange(h, h->parity);
}

void drop_graphs(cavity *h) {
  for (auto &g : h->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int build_graphs(cavity *h) {
  drop_graphs(h);
  for (int par = 0; par < 2; ++par) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_step(h, par);
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != CAVITY_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e);
    const cudaError_t e2 = cudaGraphInstantiate(&h->graph[par], g, 0);
    cudaGraphDestroy(g);
    CK(e2);
  }
  return CAVITY_OK;
}

int init_state(cavity *h) {
  CK(cudaMemsetAsync(h->d_fields, 0, h->field_bytes, h->stream));
  CK(cudaMemsetAsync(h->d_cs, 0, sizeof(CavState), h->stream));
  h->parity = 0;
  h->steps_taken = 0;
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    InitArgs a{h->d_blocks, h->d_cc, id, 0, h->desc.seed, h->desc.noise_amp, h->prm.t_hot, h->prm.t_cold};
    const long long n = (long long)B.nx * B.ny * B.nz;
    if (h->f32) k_init<float><<<ceil_div(n, 256), 256, 0, h->stream>>>(a);
    else k_init<double><<<ceil_div(n, 256), 256, 0, h->stream>>>(a);
    CK(cudaGetLastError());
  }
  return refresh_state(h);
}

// device staging buffer of at least n doubles for host transfers (grown on demand)
int ensure_stage(cavity *h, size_t n) {
  if (h->d_stage && h->stage_elems >= n) return CAVITY_OK;
  CK(cudaStreamSynchronize(h->stream));
  if (h->d_stage) {
    cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_elems = 0;
  }
  CK(cudaMalloc(&h->d_stage, n * sizeof(double)));
  h->stage_elems = n;
  return CAVITY_OK;
}

int popcount5(int m) {
  int c = 0;
  for (int f = 0; f < kNF; ++f) c += (m >> f) & 1;
  return c;
}

int read_state(cavity *h, CavState *st) {
  CK(cudaMemcpyAsync(st, h->d_cs, sizeof(CavState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int state_status(const CavState &st) {
  if (st.flags & 2) return CAVITY_ERR_TIMEOUT;
  if (st.flags & 1) return CAVITY_ERR_NONFINITE;
  return CAVITY_OK;
}

void release(cavity *h) {
  DeviceGuard g(h->dev);
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  void *ptrs[] = {h->d_fields, h->d_blocks, h->d_cc, h->d_cs, h->d_wall, h->d_cut, h->d_step_part,
                  h->d_bc_part, h->d_counter, h->d_twall, h->d_xbuf, h->d_stage, h->d_maps, h->d_nus};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

// ===========================================================================
extern "C" {

int cavity_default_params(cavity_params *p) {
  if (!p) return CAVITY_ERR_INVALID_ARG;
  p->Ra = 1e5; p->Pr = 0.71; p->cfl = 0.5; p->kappa = 0.1; p->c4 = 1.0 / 32.0;
  p->u_ref = -1.0; p->t_inf = NAN; p->t_hot = 1.0; p->t_cold = 0.0; p->gravity_axis = 2;
  resolve_defaults(p);
  return CAVITY_OK;
}

int cavity_create(const cavity_desc *desc, cavity_t **out) {
  if (!out) return CAVITY_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return CAVITY_ERR_INVALID_ARG;
  const cavity_desc &d = *desc;
  if (d.nx < 2 || d.ny < 2 || d.nz < 2 || d.px < 1 || d.py < 1 || d.pz < 1) return CAVITY_ERR_INVALID_ARG;
  if (d.nx / d.px < 2 || d.ny / d.py < 2 || d.nz / d.pz < 2) return CAVITY_ERR_INVALID_ARG;
  if ((long long)d.nx * d.ny * d.nz > (1LL << 34)) return CAVITY_ERR_INVALID_ARG;
  if (!(d.noise_amp >= 0.0) || !std::isfinite(d.noise_amp)) return CAVITY_ERR_INVALID_ARG;
  if (d.precision != CAVITY_FP64 && d.precision != CAVITY_FP32_MIXED) return CAVITY_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d.device < 0 || d.device >= ndev) return CAVITY_ERR_CUDA;
  cavity *h = new (std::nothrow) cavity();
  if (!h) return CAVITY_ERR_OOM;
  h->desc = d;
  h->dev = d.device;
  h->f32 = d.precision == CAVITY_FP32_MIXED;
  h->esize = h->f32 ? 4 : 8;
  h->na = h->f32 ? Store<float>::NA : Store<double>::NA;
  h->np = h->f32 ? Store<float>::NP : Store<double>::NP;
  if (h->f32) {
    h->tx = kF32TX;
    h->ty = kF32TY;
    h->kc = kF32KC;
    h->f32_r = kF32R;
    // tile override for tuning sweeps: BDC_F32_TILE="KC,R" (a compiled variant)
    if (const char *env = std::getenv("BDC_F32_TILE")) {
      int kc = 0, r = 0;
      if (std::sscanf(env, "%d,%d", &kc, &r) == 2 && f32_variant_ok(kc, r)) {
        h->kc = kc;
        h->f32_r = r;
      }
    }
  }
  cavity_default_params(&h->prm);
  int rc = CAVITY_OK;
  {
    DeviceGuard g(h->dev);
    if (d.stream) {
      h->stream = (cudaStream_t)d.stream;
    } else {
      if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) rc = CAVITY_ERR_CUDA;
      h->own_stream = true;
    }
    if (rc == CAVITY_OK) rc = build_layout(h);
    if (rc == CAVITY_OK) rc = alloc_device(h);
    if (rc == CAVITY_OK) rc = upload_consts(h);
    if (rc == CAVITY_OK) rc = init_state(h);
    if (rc == CAVITY_OK) rc = build_graphs(h);
    if (rc == CAVITY_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = CAVITY_ERR_CUDA;
  }
  if (rc != CAVITY_OK) {
    release(h);
    delete h;
    return rc;
  }
  *out = h;
  return CAVITY_OK;
}

int cavity_set_params(cavity_t *h, const cavity_params *p) {
  if (!h || !p) return CAVITY_ERR_INVALID_ARG;
  cavity_params q = *p;
  resolve_defaults(&q);
  if (check_params(q) != CAVITY_OK) return fail(h, CAVITY_ERR_INVALID_ARG, "invalid parameters");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  h->prm = q;
  int rc = upload_consts(h);
  if (rc != CAVITY_OK) return rc;
  if (h->steps_taken == 0) return init_state(h);
  return refresh_state(h);
}

int cavity_set_wall_temperature(cavity_t *h, int wall, const double *host, size_t n) {
  if (!h || !host || (wall != 0 && wall != 1)) return CAVITY_ERR_INVALID_ARG;
  const size_t nw = (size_t)h->desc.ny * h->desc.nz;
  if (n != nw) return fail(h, CAVITY_ERR_INVALID_ARG, "wall temperature count must be ny*nz");
  for (size_t q = 0; q < n; ++q)
    if (!std::isfinite(host[q])) return fail(h, CAVITY_ERR_INVALID_ARG, "non-finite wall temperature");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  std::copy(host, host + n, h->twall.begin() + (wall ? nw : 0));
  h->wall_custom[wall] = true;
  int rc = upload_consts(h);
  if (rc != CAVITY_OK) return rc;
  return refresh_state(h);
}

int cavity_step(cavity_t *h, int nsteps) {
  if (!h || nsteps < 0) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  for (int s = 0; s < nsteps; ++s) {
    CK(cudaGraphLaunch(h->graph[h->parity], h->stream));
    h->parity ^= 1;
    h->steps_taken += 1;
  }
  return CAVITY_OK;
}

int cavity_residual(cavity_t *h, double out[5]) {
  if (!h || !out) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  for (int f = 0; f < 5; ++f) out[f] = st.res[f];
  return state_status(st);
}

int cavity_nusselt(cavity_t *h, double *hot, double *cold) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  if (hot) *hot = st.nu_hot;
  if (cold) *cold = st.nu_cold;
  return state_status(st);
}

int cavity_get_time(cavity_t *h, long long *step, double *t, double *dt) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  if (step) *step = st.step;
  if (t) *t = st.t;
  if (dt) *dt = st.dt;
  return state_status(st);
}

int cavity_get_fields(cavity_t *h, int mask, double *host, size_t count) {
  if (!h || !host || mask <= 0 || mask > CAVITY_FIELD_ALL) return CAVITY_ERR_INVALID_ARG;
  const size_t N = (size_t)h->desc.nx * h->desc.ny * h->desc.nz;
  if (count != (size_t)popcount5(mask) * N) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    MoveArgs a{h->d_blocks, id, h->parity, mask, {h->desc.nx, h->desc.ny, h->desc.nz}, h->d_stage, st.c};
    const int grid = ceil_div((long long)B.nx * B.ny * B.nz, 256);
    if (h->f32) k_gather<float><<<grid, 256, 0, h->stream>>>(a);
    else k_gather<double><<<grid, 256, 0, h->stream>>>(a);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(host, h->d_stage, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int cavity_get_fields_box(cavity_t *h, int mask, int i0, int j0, int k0, int ni, int nj, int nk, double *host,
                          size_t count) {
  if (!h || !host || mask <= 0 || mask > CAVITY_FIELD_ALL) return CAVITY_ERR_INVALID_ARG;
  if (ni < 1 || nj < 1 || nk < 1 || i0 < 1 || j0 < 1 || k0 < 1 || i0 + ni - 1 > h->desc.nx ||
      j0 + nj - 1 > h->desc.ny || k0 + nk - 1 > h->desc.nz)
    return fail(h, CAVITY_ERR_INVALID_ARG, "box outside the interior");
  const size_t n = (size_t)ni * nj * nk;
  if (count != (size_t)popcount5(mask) * n) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  BoxArgs a{h->d_blocks, h->nblocks, h->parity, mask, i0, j0, k0, ni, nj, nk, h->d_stage, st.c};
  if (h->f32) k_gather_box<float><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(a);
  else k_gather_box<double><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(a);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host, h->d_stage, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int cavity_set_fields(cavity_t *h, int mask, const double *host, size_t count) {
  if (!h || !host || mask <= 0 || mask > CAVITY_FIELD_ALL) return CAVITY_ERR_INVALID_ARG;
  const size_t N = (size_t)h->desc.nx * h->desc.ny * h->desc.nz;
  if (count != (size_t)popcount5(mask) * N) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  // fold the pending centre shift into the stored p, then c = 0
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    if (st.c != 0.0 && !(mask & CAVITY_FIELD_P)) {
      const int grid = ceil_div((long long)(B.nx + 4) * (B.ny + 4) * (B.nz + 4), 256);
      if (h->f32) k_shift_p<float><<<grid, 256, 0, h->stream>>>(h->d_blocks, id, h->parity, st.c);
      else k_shift_p<double><<<grid, 256, 0, h->stream>>>(h->d_blocks, id, h->parity, st.c);
      CK(cudaGetLastError());
    }
  }
  CK(cudaMemsetAsync(&h->d_cs->c, 0, sizeof(double), h->stream));
  CK(cudaMemcpyAsync(h->d_stage, host, count * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    MoveArgs a{h->d_blocks, id, h->parity, mask, {h->desc.nx, h->desc.ny, h->desc.nz}, h->d_stage, 0.0};
    const int grid = ceil_div((long long)B.nx * B.ny * B.nz, 256);
    if (h->f32) k_scatter<float><<<grid, 256, 0, h->stream>>>(a);
    else k_scatter<double><<<grid, 256, 0, h->stream>>>(a);
    CK(cudaGetLastError());
  }
  rc = refresh_state(h);
  if (rc != CAVITY_OK) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int cavity_num_blocks(cavity_t *h) { return h ? h->nblocks : CAVITY_ERR_INVALID_ARG; }

int cavity_get_block_array(cavity_t *h, int block, int field, double *host, size_t count, int dims[6]) {
  if (!h || block < 0 || block >= h->nblocks || field < 0 || field >= h->na) return CAVITY_ERR_INVALID_ARG;
  const BlockDev &B = h->hb[block];
  const size_t n = (size_t)(B.nx + 4) * (B.ny + 4) * (B.nz + 4);
  if (dims) { dims[0] = B.nx; dims[1] = B.ny; dims[2] = B.nz; dims[3] = B.ox; dims[4] = B.oy; dims[5] = B.oz; }
  if (!host) return count == 0 ? CAVITY_OK : CAVITY_ERR_INVALID_ARG;
  if (count != n) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  if (h->f32) k_copy_block<float><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(h->d_blocks, block, h->parity, field, h->d_stage);
  else k_copy_block<double><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(h->d_blocks, block, h->parity, field, h->d_stage);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host, h->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int cavity_get_face_buffer(cavity_t *h, int block, int face, double *host, size_t count) {
  if (!h || !host || block < 0 || block >= h->nblocks || face < 0 || face > 5) return CAVITY_ERR_INVALID_ARG;
  for (const CutFace &c : h->hcut) {
    if (c.src != block || c.face != face) continue;
    const size_t n = (size_t)(2 * h->np + 4) * c.nb * c.nc;
    if (count != n) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
    DeviceGuard g(h->dev);
    if (h->f32) {
      std::vector<float> tmp(n);
      CK(cudaMemcpyAsync(tmp.data(), (float *)h->d_xbuf + c.buf_off, n * sizeof(float), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (size_t q = 0; q < n; ++q) host[q] = (double)tmp[q];
    } else {
      CK(cudaMemcpyAsync(host, (double *)h->d_xbuf + c.buf_off, n * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    return CAVITY_OK;
  }
  return fail(h, CAVITY_ERR_INVALID_ARG, "face is a wall");
}

int cavity_exchange(cavity_t *h) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  return launch_exchange(h, h->parity);
}

int cavity_time_kernels(cavity_t *h, int nsteps, double ms[4]) {
  if (!h || !ms || nsteps < 1) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  cudaEvent_t ev[5];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  double acc[4] = {0, 0, 0, 0};
  int rc = CAVITY_OK;
  for (int s = 0; s < nsteps && rc == CAVITY_OK; ++s) {
    const int par = h->parity;
    cudaEventRecord(ev[0], h->stream);
    launch_step_kernel(h, par);
    cudaEventRecord(ev[1], h->stream);
    launch_bc_kernel(h, par ^ 1, 0);
    cudaEventRecord(ev[2], h->stream);
    if (h->n_cut > 0) launch_pack(h, par ^ 1);
    cudaEventRecord(ev[3], h->stream);
    if (h->n_cut > 0) launch_unpack(h, par ^ 1);
    cudaEventRecord(ev[4], h->stream);
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { rc = fail(h, CAVITY_ERR_CUDA, cudaGetErrorString(e)); break; }
    for (int q = 0; q < 4; ++q) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      acc[q] += t;
    }
    h->parity ^= 1;
    h->steps_taken += 1;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int q = 0; q < 4; ++q) ms[q] = acc[q] / nsteps;
  if (h->n_cut == 0) ms[2] = ms[3] = 0.0;
  return rc;
}

int cavity_sync(cavity_t *h) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, &st);
  if (rc != CAVITY_OK) return rc;
  return state_status(st);
}

int cavity_destroy(cavity_t *h) {
  if (!h) return CAVITY_OK;
  release(h);
  delete h;
  return CAVITY_OK;
}

const char *cavity_strerror(int code) {
  switch (code) {
    case CAVITY_OK: return "ok";
    case CAVITY_ERR_INVALID_ARG: return "invalid argument";
    case CAVITY_ERR_OOM: return "out of memory";
    case CAVITY_ERR_CUDA: return "CUDA runtime error";
    case CAVITY_ERR_NONFINITE: return "non-finite residual or spectral radius";
    case CAVITY_ERR_TIMEOUT: return "device-side wait timed out";
    case CAVITY_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char *cavity_last_error(cavity_t *h) { return h ? h->err.c_str() : ""; }

}  // extern "C"
