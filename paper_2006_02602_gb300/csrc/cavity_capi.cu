// C ABI of the buoyancy-driven-cavity step (include/cavity.h): host runtime
// that lays out the blocks of one or many cavities in HBM, builds the work
// lists of the kernels in bdc_device.cuh / bdc_step_f32.cuh, captures one CUDA
// graph per buffer parity and replays it.  Two arithmetic forms share the
// runtime: FP64 (five FP64 arrays per buffer set) and FP32-mixed (p_hi, p_lo,
// u, v, w, T in FP32, read by the step kernel through TMA tensor maps).  A
// handle holds either one cavity split into blocks (Section 3.2
// decomposition) or a batch of single-block cavities.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cfloat>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cavity.h"
#include "bdc_adjoint.cuh"
#include "bdc_device.cuh"
#include "bdc_step_f32.cuh"

using namespace bdc;

namespace {

// k_step tile of the FP64 form: 32 x 4 threads (166 registers each: three
// CTAs, 12 warps, per SM hide the FP64 pipe's latency better than one CTA of
// 32 x 8), 8-plane chunks
constexpr int kTX = 32, kTY = 4, kKC = 8;

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

std::vector<int> split_sizes(int n, int parts) {  // Section 3.2: as even as possible
  std::vector<int> s(parts, n / parts);
  for (int r = 0; r < n % parts; ++r) s[r] += 1;
  return s;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// FP32 step-kernel variants compiled in: (kernel form P, tile height TY, ring
// depth R); P = 3 is k_step_f32q (two nodes per thread, the nodes behind the
// plane in registers), the one form.  The z-chunk depth is a run-time
// parameter of the tiling (the autotuner tries kF32Chunks).
#define BDC_F32_VARIANTS(X) X(3, 8, 4) X(3, 8, 5) X(3, 16, 4) X(3, 16, 5)
struct F32Shape {
  int p, ty, kc, r;
};
const int kF32Chunks[] = {16, 24, 32, 40, 48, 64, 96};
constexpr int kF32MaxChunk = 4096;

bool f32_variant_ok(int p, int ty, int kc, int r) {
  if (kc < 1 || kc > kF32MaxChunk) return false;
#define BDC_OK(P, TY, R) \
  if (p == P && ty == TY && r == R) return true;
  BDC_F32_VARIANTS(BDC_OK)
#undef BDC_OK
  return false;
}

// every (variant, chunk depth) pair the autotuner times
std::vector<F32Shape> f32_shapes() {
  std::vector<F32Shape> out;
#define BDC_SHAPE(P, TY, R) \
  for (int kc : kF32Chunks) out.push_back({P, TY, kc, R});
  BDC_F32_VARIANTS(BDC_SHAPE)
#undef BDC_SHAPE
  return out;
}

}  // namespace

// checkpoints and work arrays of the discrete adjoint (single-block cavity)
struct AdjointStore {
  int nsteps = 0, ckpt = 0, ncp = 0, nparts = 0;
  size_t set_bytes = 0;        // one buffer set of the block
  char *ckpt_mem = nullptr;    // ncp buffer sets: the state at steps 0, ckpt, 2 ckpt, ...
  CavState *ckpt_cs = nullptr;  // their scalars (device)
  char *seg_mem = nullptr;     // ckpt buffer sets: one recomputed segment
  BlockDev *seg_blocks = nullptr;   // ckpt block descriptors, slot s's state as buffer set 0 (walls pass)
  WallFace *seg_faces = nullptr;    // the block's wall faces once per slot (one walls launch per segment)
  CUtensorMap *seg_maps = nullptr;  // FP32 form: the step kernel's two maps of every slot
  char *final_mem = nullptr;   // the state after the forward run
  CavState final_cs{};
  int final_parity = 0;
  long long final_steps = 0;
  void *X = nullptr, *Yt = nullptr, *Q = nullptr;  // adjoint arrays: FP64 (FP64 forward) or FP32 (FP32-mixed)
  double *thetabar = nullptr, *scal = nullptr, *argpart = nullptr;
  double *gpart = nullptr;     // per-CTA node sums of the FP32 gather (3 per CTA)
  double *dts = nullptr;       // dt of every step (device)
  unsigned int *cnt = nullptr; // finished CTAs of k_adj_pre (zero between launches)
  BlockDev *block = nullptr;   // descriptor of a segment slot (wall pass of FP32 states)
  bool have_forward = false;
  double J = 0.0;
};

struct cavity {
  int dev = 0;
  bool u_ref_auto = true;  // u_ref follows Ra (default)
  AdjointStore adj;
  std::vector<cudaEvent_t> adj_ev;  // two per reverse step: around the rates' reverse kernel
  double adj_rates_ms = 0.0;        // its mean duration in the last reverse sweep
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int ncav = 1;
  std::vector<cavity_desc> descs;
  std::vector<cavity_params> prms;
  std::vector<CavConst> hcc;
  std::vector<char> wall_custom;  // 2 per cavity
  std::vector<double> twall;      // per cavity: hot wall then cold wall (ny*nz each) at wall_off
  bool f32 = false;               // FP32-mixed form
  size_t esize = 8;               // bytes per stored element
  int na = 5;                     // stored arrays per buffer set
  int np = 1;                     // pressure arrays
  int tx = kTX, ty = kTY, kc = kKC;
  int f32_r = 0;                  // ring depth of the FP32 step kernel
  int f32_p = 1;                  // nodes per thread along x of the FP32 step kernel
  int local_dt = 0;               // CAVITY_DT_LOCAL: each node at its own stable step
  long long wait_cycles = kWaitCycles;  // limit of the FP32 step kernel's bounded waits
  int withhold_plane = -1;              // timeout test: tile plane whose load is not issued
  // interior/shell split with overlapped exchange (FP64, single cavity, cut faces)
  bool overlap = false;
  std::vector<ShellFace> hshell;
  ShellFace *d_shell = nullptr;
  int n_shell = 0;                // k_shell_f64 CTAs
  cudaStream_t side = nullptr;    // the exchange's stream while the interior is stepped
  cudaEvent_t ev_shell = nullptr, ev_exch = nullptr;
  int nblocks = 0;
  std::vector<BlockDev> hb;
  std::vector<WallFace> hwall;
  std::vector<CutFace> hcut;
  long long xbuf_elems = 0;
  int n_step = 0, n_bc = 0, n_cut = 0;
  int nslices = kFinSlices;  // k_finalize CTAs per cavity: about 128 step partials a slice
  int n_coarse = 0;  // FP64 step tiles of KC planes (scheduled before the fine ones)
  int part_cap = 0;  // step partials allocated (CTAs)

  BlockDev *d_blocks = nullptr;
  CavConst *d_cc = nullptr;
  CavState *d_cs = nullptr;
  WallFace *d_wall = nullptr;
  CutFace *d_cut = nullptr;
  CUtensorMap *d_maps = nullptr;
  double *d_step_part = nullptr, *d_bc_part = nullptr, *d_twall = nullptr, *d_stage = nullptr;
  double *d_fin = nullptr;  // k_finalize slice totals [ncav][kFinSlices][8]
  StepRecord *d_log = nullptr;  // the step log (device address of caller-owned host memory), or null
  long long log_cap = 0;
  unsigned int *d_counter = nullptr;  // [ncav] k_bc CTAs done per cavity, the FP64 step's tile counter,
                                      // [ncav] the FP64 step's dt-filter floors
  int persist_ctas = 0;               // CTAs of the persistent FP64 step kernel that fit on the GPU
  void *d_fields = nullptr, *d_xbuf = nullptr;
  size_t field_bytes = 0;
  size_t stage_elems = 0;

  int parity = 0;
  long long steps_taken = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step from parity 0 / 1
  cudaGraphExec_t graph2[2] = {nullptr, nullptr};  // two steps from parity 0 / 1 (programmatic edge between them)
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

void fill_consts(cavity *h, int c) {
  const int gn[3] = {h->descs[c].nx, h->descs[c].ny, h->descs[c].nz};
  set_cav_physics(h->hcc[c], gn, h->prms[c]);
}

void resolve_defaults(cavity_params *p) {
  if (!(p->u_ref >= 0.0)) p->u_ref = std::max(1.0, std::sqrt(p->Ra * p->Pr));
  if (std::isnan(p->t_inf)) p->t_inf = 0.5 * (p->t_hot + p->t_cold);
}

int check_params(const cavity_params &p) {
  if (!(p.Ra >= 0.0) || !(p.Pr > 0.0) || !(p.cfl > 0.0) || !(p.kappa > 0.0) || !(p.c4 >= 0.0) ||
      !(p.u_ref > 0.0) || !(p.kappa * p.u_ref * p.u_ref >= FLT_MIN) ||
      !(p.kappa * p.u_ref * p.u_ref < 1e300) || !std::isfinite(p.t_inf) || !std::isfinite(p.t_hot) || !std::isfinite(p.t_cold) ||
      p.t_hot == p.t_cold || (p.gravity_axis != 1 && p.gravity_axis != 2))
    return CAVITY_ERR_INVALID_ARG;
  return CAVITY_OK;
}

int check_desc(const cavity_desc &d) {
  if (d.nx < 2 || d.ny < 2 || d.nz < 2 || d.px < 1 || d.py < 1 || d.pz < 1) return CAVITY_ERR_INVALID_ARG;
  if (d.nx / d.px < 2 || d.ny / d.py < 2 || d.nz / d.pz < 2) return CAVITY_ERR_INVALID_ARG;
  if ((long long)d.nx * d.ny * d.nz > (1LL << 34)) return CAVITY_ERR_INVALID_ARG;
  if (!(d.noise_amp >= 0.0) || !std::isfinite(d.noise_amp)) return CAVITY_ERR_INVALID_ARG;
  if (d.precision != CAVITY_FP64 && d.precision != CAVITY_FP32_MIXED) return CAVITY_ERR_INVALID_ARG;
  return CAVITY_OK;
}

// ---------------------------------------------------------------------------
// layout: blocks of every cavity, wall / cut face lists, centre nodes

// Step-kernel tiles and their partial slots, block by block (a cavity's
// slots are contiguous).  The planes below the last KC-plane boundary go in
// KC-plane chunks, the rest in fine chunks scheduled after every block's
// coarse tiles: kFineKC planes in the FP64 form; kFineKC32 planes in the
// FP32 form, and only in blocks deeper than one chunk (a shallower block is
// one chunk: the ring's fill is paid per tile).
void assign_tiles(cavity *h) {
  int tile = 0, coarse = 0, fine = 0;
  for (int c = 0; c < h->ncav; ++c) h->hcc[c].tile_begin = -1;
  for (BlockDev &B : h->hb) {
    B.tiles_x = ceil_div(B.nx, h->tx);
    B.tiles_y = ceil_div(B.ny, h->ty);
    const int kf = h->f32 ? kFineKC32 : kFineKC;
    if (h->f32 && B.nz <= h->kc) {
      B.tiles_zc = 1;
      B.zsplit = B.nz;
    } else {
      B.tiles_zc = (B.nz - 1) / h->kc;
      B.zsplit = B.tiles_zc * h->kc;
    }
    B.tiles_z = B.tiles_zc + ceil_div(B.nz - B.zsplit, kf);
    B.tile_begin = tile;
    B.coarse_begin = coarse;
    B.fine_begin = fine;
    CavConst &C = h->hcc[B.cav];
    if (C.tile_begin < 0) C.tile_begin = tile;
    tile += B.tiles_x * B.tiles_y * B.tiles_z;
    coarse += B.tiles_x * B.tiles_y * B.tiles_zc;
    fine += B.tiles_x * B.tiles_y * (B.tiles_z - B.tiles_zc);
    C.tile_end = tile;
  }
  h->n_step = tile;
  h->n_coarse = coarse;
  int most = 0;  // the most tiles of one cavity
  for (int c = 0; c < h->ncav; ++c) most = std::max(most, h->hcc[c].tile_end - h->hcc[c].tile_begin);
  h->nslices = std::max(1, std::min(kFinSlices, ceil_div(most, 128)));
  for (int c = 0; c < h->ncav; ++c) {  // contiguous slices of each cavity's step partials
    CavConst &C = h->hcc[c];
    const long long nt = C.tile_end - C.tile_begin;
    for (int g = 0; g <= kFinSlices; ++g)
      C.slice_q[g] = C.tile_begin + (int)(nt * std::min(g, h->nslices) / h->nslices);
  }
}

int build_layout(cavity *h) {
  const size_t es = h->esize;
  const int row_align = (int)(128 / es);
  h->hb.clear();
  size_t total_elems = 0;
  long long wall_off = 0;
  for (int cv = 0; cv < h->ncav; ++cv) {
    const cavity_desc &d = h->descs[cv];
    const int pg[3] = {d.px, d.py, d.pz};
    const int gn[3] = {d.nx, d.ny, d.nz};
    std::vector<int> sz[3], org[3];
    for (int a = 0; a < 3; ++a) {
      sz[a] = split_sizes(gn[a], pg[a]);
      int o = 0;
      for (int s : sz[a]) { org[a].push_back(o); o += s; }
    }
    const int first = (int)h->hb.size();
    for (int bz = 0; bz < pg[2]; ++bz)
      for (int by = 0; by < pg[1]; ++by)
        for (int bx = 0; bx < pg[0]; ++bx) {
          BlockDev B{};
          B.nx = sz[0][bx]; B.ny = sz[1][by]; B.nz = sz[2][bz];
          B.ox = org[0][bx]; B.oy = org[1][by]; B.oz = org[2][bz];
          B.pitch = ((xo1(es) + B.nx + 2 + row_align - 1) / row_align) * row_align;
          B.rows = B.ny + 4;
          B.plane = (long long)B.pitch * B.rows;
          B.fstride = ((B.plane * (B.nz + 4) + 63) / 64) * 64;
          const int c3[3] = {bx, by, bz};
          for (int f = 0; f < 6; ++f) {
            const int a = f / 2, hi = f % 2;
            int cc[3] = {c3[0], c3[1], c3[2]};
            cc[a] += hi ? 1 : -1;
            const bool inside = cc[a] >= 0 && cc[a] < pg[a];
            B.wall[f] = inside ? 0 : 1;
            B.nbr[f] = inside ? first + cc[0] + pg[0] * (cc[1] + pg[1] * cc[2]) : -1;
          }
          B.cav = cv;
          h->hb.push_back(B);
          total_elems += 2 * (size_t)h->na * (size_t)B.fstride;
        }
    CavConst &C = h->hcc[cv];
    C.wall_off = wall_off;
    wall_off += 2LL * d.ny * d.nz;
    // centre nodes in (k, j, i) lexicographic order
    std::vector<int> ax[3];
    for (int a = 0; a < 3; ++a) {
      if (gn[a] % 2 == 1) ax[a] = {(gn[a] + 1) / 2};
      else ax[a] = {gn[a] / 2, gn[a] / 2 + 1};
    }
    int m = 0;
    for (int K : ax[2])
      for (int J : ax[1])
        for (int I : ax[0]) {
          for (int id = first; id < (int)h->hb.size(); ++id) {
            const BlockDev &B = h->hb[id];
            if (I > B.ox && I <= B.ox + B.nx && J > B.oy && J <= B.oy + B.ny && K > B.oz && K <= B.oz + B.nz) {
              C.centre_blk[m] = id;
              C.centre_off[m] = host_node_index(B, es, I - B.ox, J - B.oy, K - B.oz);
            }
          }
          ++m;
        }
    C.ncentre = m;
  }
  h->nblocks = (int)h->hb.size();
  h->field_bytes = total_elems * es;
  h->twall.assign((size_t)wall_off, 0.0);
  assign_tiles(h);
  // wall faces, contiguous per cavity, and cut faces, each list with its x
  // faces first: a CTA of an x face touches one 32-byte sector per node and
  // array (its positions run along y) where the others' rows are contiguous,
  // and launched first the x faces' CTAs spread over the SMs (after a 128^3
  // FP32 step in 2 x 2 x 2 blocks the last exchange CTA ended 14-15 us after
  // the step kernel with the faces in block order, 10-12 us in this order
  // together with the finalise's reduction trees)
  h->hwall.clear();
  h->hcut.clear();
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    const int n[3] = {B.nx, B.ny, B.nz};
    for (int f = 0; f < 6; ++f) {
      const int a = f / 2;
      const int n1 = n[a == 0 ? 1 : 0], n2 = n[a == 2 ? 1 : 2];
      if (B.wall[f]) h->hwall.push_back(WallFace{id, f, n1, n2, 0, B.cav});
      else h->hcut.push_back(CutFace{id, f, B.nbr[f], n1, n2, 0, 0});
    }
  }
  std::stable_sort(h->hwall.begin(), h->hwall.end(), [](const WallFace &x, const WallFace &y) {
    return x.cav != y.cav ? x.cav < y.cav : x.face / 2 < y.face / 2;
  });
  std::stable_sort(h->hcut.begin(), h->hcut.end(),
                   [](const CutFace &x, const CutFace &y) { return x.face / 2 < y.face / 2; });
  int bc = 0, cut = 0;
  long long xoff = 0;
  for (int c = 0; c < h->ncav; ++c) h->hcc[c].bc_begin = -1;
  for (WallFace &w : h->hwall) {
    CavConst &C = h->hcc[w.cav];
    w.cta_begin = bc;
    if (C.bc_begin < 0) C.bc_begin = C.bc_xend = bc;
    bc += ceil_div((long long)w.n1 * w.n2, kBcThreads);
    C.bc_end = bc;
    if (w.face / 2 == 0) C.bc_xend = bc;
  }
  for (CutFace &c : h->hcut) {
    c.cta_begin = cut;
    c.buf_off = xoff;
    cut += ceil_div((long long)c.nb * c.nc, 256);
    xoff += (long long)(h->na + h->np) * c.nb * c.nc;
  }
  h->n_bc = bc;
  h->n_cut = cut;
  h->xbuf_elems = xoff;
  return CAVITY_OK;
}

// TMA descriptors of the FP32-mixed step kernel: two 4-D maps per block and
// buffer set over (x, y, z, array): the pressure box (40 x (TY+4) nodes of
// p_hi and p_lo) and the box of the other five arrays (40 x (TY+2) nodes)
// The pressure-box and other-box maps (out[0], out[1]) of a buffer set of
// block B's layout at `base`.
int encode_block_maps(cavity *h, const BlockDev &B, void *base, CUtensorMap out[2]) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) return fail(h, CAVITY_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  EncodeTiledFn encode = (EncodeTiledFn)fn;
  for (int kind = 0; kind < 2; ++kind) {
    // columns up to node nx + 2: the row's padding lies outside the map, so a
    // box reaching past it is zero-filled, not read from HBM
    const cuuint64_t dims[4] = {(cuuint64_t)(XO<float>::v + B.nx + 2), (cuuint64_t)B.rows, (cuuint64_t)(B.nz + 4),
                                (cuuint64_t)kF32NA};
    const cuuint64_t strides[3] = {(cuuint64_t)B.pitch * 4, (cuuint64_t)B.plane * 4, (cuuint64_t)B.fstride * 4};
    const cuuint32_t box[4] = {(cuuint32_t)kF32BX, (cuuint32_t)(kind == 0 ? f32_box_yp(h->ty) : f32_box_yo(h->ty)), 1,
                               (cuuint32_t)(kind == 0 ? kF32NP : kF32NO)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&out[kind], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, CAVITY_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  }
  return CAVITY_OK;
}

int encode_maps(cavity *h) {
  std::vector<CUtensorMap> maps(4 * h->nblocks);
  for (int id = 0; id < h->nblocks; ++id)
    for (int s = 0; s < 2; ++s) {
      const int rc = encode_block_maps(h, h->hb[id], h->hb[id].base[s], &maps[2 * (2 * id + s)]);
      if (rc != CAVITY_OK) return rc;
    }
  if (!h->d_maps) CK(cudaMalloc(&h->d_maps, sizeof(CUtensorMap) * maps.size()));
  CK(cudaMemcpy(h->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
  return CAVITY_OK;
}

template <int P, int TY, int R>
auto f32_kernel() {
  static_assert(P == 3, "the FP32 step kernel has one form");
  return k_step_f32q<TY, R>;
}

// dynamic shared memory of the FP32 step kernel's shape, and the largest
// shared-memory carveout (four 47 KB CTAs per SM)
cudaError_t f32_set_smem(int p, int ty, int r) {
#define BDC_ATTR(P, TY, R)                                                                                       \
  if (p == P && ty == TY && r == R) {                                                                            \
    const cudaError_t e = cudaFuncSetAttribute(f32_kernel<P, TY, R>(),                                           \
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, f32_smem_bytes(TY, R)); \
    if (e != cudaSuccess) return e;                                                                              \
    return cudaFuncSetAttribute(f32_kernel<P, TY, R>(), cudaFuncAttributePreferredSharedMemoryCarveout,         \
                                (int)cudaSharedmemCarveoutMaxShared);                                            \
  }
  BDC_F32_VARIANTS(BDC_ATTR)
#undef BDC_ATTR
  return cudaErrorInvalidValue;
}

int upload_tables(cavity *h) {
  CK(cudaMemcpyAsync(h->d_blocks, h->hb.data(), sizeof(BlockDev) * h->nblocks, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_cc, h->hcc.data(), sizeof(CavConst) * h->ncav, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int ensure_partials(cavity *h) {
  const int need = h->n_step + (h->overlap ? h->n_shell : 0);
  if (h->part_cap >= need) return CAVITY_OK;
  CK(cudaStreamSynchronize(h->stream));
  if (h->d_step_part) cudaFree(h->d_step_part);
  h->d_step_part = nullptr;
  CK(cudaMalloc(&h->d_step_part, sizeof(double) * kPartStride * std::max(1, need)));
  h->part_cap = need;
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
  CK(cudaMalloc(&h->d_cc, sizeof(CavConst) * h->ncav));
  CK(cudaMalloc(&h->d_cs, sizeof(CavState) * h->ncav));
  CK(cudaMemsetAsync(h->d_cs, 0, sizeof(CavState) * h->ncav, h->stream));
  CK(cudaMalloc(&h->d_wall, sizeof(WallFace) * std::max<size_t>(1, h->hwall.size())));
  CK(cudaMalloc(&h->d_cut, sizeof(CutFace) * std::max<size_t>(1, h->hcut.size())));
  int rc = ensure_partials(h);
  if (rc != CAVITY_OK) return rc;
  CK(cudaMalloc(&h->d_bc_part, sizeof(double) * 2 * std::max(1, h->n_bc)));
  CK(cudaMalloc(&h->d_fin, sizeof(double) * 8 * kFinSlices * h->ncav));
  CK(cudaMalloc(&h->d_counter, sizeof(unsigned int) * (2 * h->ncav + 1)));
  CK(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned int) * (2 * h->ncav + 1), h->stream));
  {
    int nsm = 0, per_sm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev));
    if (h->ty == 4)
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_f64<kTX, 4, kKC>, kTX * 4, 0));
    else
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_f64<kTX, 8, kKC>, kTX * 8, 0));
    h->persist_ctas = std::max(1, nsm * per_sm);
  }
  CK(cudaMalloc(&h->d_twall, sizeof(double) * std::max<size_t>(1, h->twall.size())));
  if (h->xbuf_elems > 0) CK(cudaMalloc(&h->d_xbuf, h->esize * (size_t)h->xbuf_elems));
  if (!h->hwall.empty())
    CK(cudaMemcpyAsync(h->d_wall, h->hwall.data(), sizeof(WallFace) * h->hwall.size(), cudaMemcpyHostToDevice, h->stream));
  if (!h->hcut.empty())
    CK(cudaMemcpyAsync(h->d_cut, h->hcut.data(), sizeof(CutFace) * h->hcut.size(), cudaMemcpyHostToDevice, h->stream));
  if (h->f32) {
    rc = encode_maps(h);
    if (rc != CAVITY_OK) return rc;
    CK(f32_set_smem(h->f32_p, h->ty, h->f32_r));
  }
  return CAVITY_OK;
}

int upload_consts(cavity *h) {
  for (int c = 0; c < h->ncav; ++c) {
    fill_consts(h, c);
    const size_t nw = (size_t)h->descs[c].ny * h->descs[c].nz;
    double *tw = h->twall.data() + h->hcc[c].wall_off;
    if (!h->wall_custom[2 * c]) std::fill(tw, tw + nw, h->prms[c].t_hot);
    if (!h->wall_custom[2 * c + 1]) std::fill(tw + nw, tw + 2 * nw, h->prms[c].t_cold);
  }
  int rc = upload_tables(h);
  if (rc != CAVITY_OK) return rc;
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
  a.tile_counter = h->d_counter + h->ncav; a.ntiles = h->n_step; a.local_dt = h->local_dt;
  a.sfloor = h->d_counter + h->ncav + 1;
  a.ncoarse = h->n_coarse;
  a.skip_shell = 0;
  return a;
}

StepF32Args step_f32_args(cavity *h, int parity) {
  StepF32Args a;
  a.blocks = h->d_blocks; a.nblocks = h->nblocks; a.cc = h->d_cc; a.cs = h->d_cs;
  a.maps = h->d_maps; a.partials = h->d_step_part; a.parity = parity; a.local_dt = h->local_dt;
  a.ncoarse = h->n_coarse;
  a.wait_cycles = h->wait_cycles;
  a.withhold_plane = h->withhold_plane;
  a.ghosts_late = h->n_cut > 0;  // the finalise after each step writes the ghost layers
  return a;
}

BcArgs bc_args(cavity *h, int parity, int mode) {
  BcArgs a;
  a.blocks = h->d_blocks;
  a.faces = h->d_wall;
  a.nfaces = (int)h->hwall.size();
  a.cc = h->d_cc; a.cs = h->d_cs; a.ncav = h->ncav;
  a.step_partials = h->d_step_part; a.bc_partials = h->d_bc_part; a.counter = h->d_counter;
  a.tile_counter = h->d_counter + h->ncav;
  a.sfloor = h->d_counter + h->ncav + 1;
  a.t_wall = h->d_twall; a.parity = parity; a.mode = mode;
  a.shell_begin = a.shell_end = 0;
  a.log = mode == 1 || mode == 3 ? nullptr : h->d_log;  // after a step (modes 0, 4): the step log
  a.log_cap = h->log_cap;
  a.cuts = nullptr; a.ncuts = 0; a.xbuf = nullptr;
  a.nslices = h->nslices;
  a.wall_ctas = 0;
  return a;
}

ExchArgs exch_args(cavity *h, int parity) {
  ExchArgs a;
  a.blocks = h->d_blocks; a.faces = h->d_cut; a.nfaces = (int)h->hcut.size();
  a.buf = (double *)h->d_xbuf; a.parity = parity;
  return a;
}

// The persistent FP64 step kernel of the handle's tile height (8 or 4 rows;
// 32 x TY threads, as many CTAs as fit on the GPU at once).
void launch_step_f64(cavity *h, const StepArgs &a) {
  const int grid = std::min(h->n_step, h->persist_ctas);
  if (h->ty == 4)
    k_step_f64<kTX, 4, kKC><<<grid, dim3(kTX, 4), 0, h->stream>>>(a);
  else
    k_step_f64<kTX, 8, kKC><<<grid, dim3(kTX, 8), 0, h->stream>>>(a);
}

// `after_finalise`: the launch directly follows, in the same stream capture,
// the finalise of the previous step (the second step of a two-step graph).
// The FP32 step kernel is then launched as a programmatic dependent: its
// prologue (TMA loads of the state, which the previous step kernel completed
// before that finalise started) overlaps the finalise, and it waits for the
// finalise before reading dt and the centre shift.  With cut faces that
// finalise also exchanges the ghost layers, so a tile whose boxes reach a
// ghost layer waits for it before its first load.  Every other predecessor
// (an unpack writing ghost layers, a state upload, a copy) gets a plain
// launch.
void launch_step_kernel(cavity *h, int parity, bool after_finalise = false) {
  if (h->f32) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->n_step);
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = after_finalise ? 1 : 0;
    const StepF32Args sa = step_f32_args(h, parity);
#define BDC_LAUNCH(P, TY, R)                                                     \
  if (h->f32_p == P && h->ty == TY && h->f32_r == R) {                            \
    cfg.blockDim = dim3(kF32TX / 2, TY);                                          \
    cfg.dynamicSmemBytes = f32_smem_bytes(TY, R);                                 \
    cudaLaunchKernelEx(&cfg, f32_kernel<P, TY, R>(), sa);                         \
  }
    BDC_F32_VARIANTS(BDC_LAUNCH)
#undef BDC_LAUNCH
  } else {
    launch_step_f64(h, step_args(h, parity, 0));
  }
}

void launch_spectral(cavity *h) {
  const StepArgs sa = step_args(h, h->parity, 1);
  if (h->f32) {
#define BDC_SPEC(P, TY, R)                                                                                       \
  if (h->f32_p == P && h->ty == TY && h->f32_r == R)                                                             \
    k_spectral<float, kF32TX, TY><<<h->n_step, dim3(kF32TX, TY), 0, h->stream>>>(sa);
    BDC_F32_VARIANTS(BDC_SPEC)
#undef BDC_SPEC
  } else {
    launch_step_f64(h, sa);
  }
}

// mode 0: after a step; mode 1: state refresh; 3: walls only.  The walls
// kernel (k_bc) writes the walls and the Nusselt partials, k_finalize reduces
// the partials and advances the state; after an FP64 step the wall CTAs run
// inside the finalise launch, arriving at each cavity's completion counter
// with the finalise CTAs, and the last to arrive folds their partials.  The
// FP32 step kernel applies the walls where it reads them and leaves the
// Nusselt sums in its own partials, so after its steps only k_finalize
// runs.  After a step of a decomposed
// cavity the finalise launch carries one more CTA per 256 cut-face
// positions, which exchange the new state's cut faces (Section 4.5 pack and
// unpack in one pass) beside the reductions: one launch after the step
// instead of a finalise beside a pack and an unpack.
void launch_bc_kernel(cavity *h, int parity, int mode) {
  const int nfin = h->ncav * h->nslices;
  BcArgs b = bc_args(h, parity, h->f32 && mode == 0 ? 4 : mode);
  int grid = nfin;
  if (mode == 0 && !h->f32) {  // the FP64 walls and their Nusselt partials in the same launch
    b.wall_ctas = h->n_bc;
    grid += h->n_bc;
  }
  if (mode == 0 && h->n_cut > 0) {
    b.cuts = h->d_cut;
    b.ncuts = (int)h->hcut.size();
    b.xbuf = h->d_xbuf;
    grid += h->n_cut;
  }
  if (h->f32) {
    if (mode == 0) {
      k_finalize<float><<<grid, kFinThreads, 0, h->stream>>>(b, h->d_fin);
      return;
    }
    k_bc<float><<<h->n_bc, kBcThreads, 0, h->stream>>>(bc_args(h, parity, mode));
    if (mode != 3) k_finalize<float><<<nfin, kFinThreads, 0, h->stream>>>(bc_args(h, parity, mode), h->d_fin);
  } else {
    if (mode == 0) {
      k_finalize<double><<<grid, kFinThreads, 0, h->stream>>>(b, h->d_fin);
      return;
    }
    k_bc<double><<<h->n_bc, kBcThreads, 0, h->stream>>>(bc_args(h, parity, mode));
    if (mode != 3) k_finalize<double><<<nfin, kFinThreads, 0, h->stream>>>(b, h->d_fin);
  }
}

void launch_pack(cavity *h, int parity, cudaStream_t s = nullptr) {
  if (!s) s = h->stream;
  if (h->f32) k_pack<float><<<h->n_cut, 256, 0, s>>>(exch_args(h, parity));
  else k_pack<double><<<h->n_cut, 256, 0, s>>>(exch_args(h, parity));
}

void launch_unpack(cavity *h, int parity, cudaStream_t s = nullptr) {
  if (!s) s = h->stream;
  if (h->f32) k_unpack<float><<<h->n_cut, 256, 0, s>>>(exch_args(h, parity));
  else k_unpack<double><<<h->n_cut, 256, 0, s>>>(exch_args(h, parity));
}

int launch_exchange(cavity *h, int parity) {
  if (h->n_cut == 0) return CAVITY_OK;
  launch_pack(h, parity);
  CK(cudaGetLastError());
  launch_unpack(h, parity);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// The overlapped step (FP64, cut faces): shell nodes first, then the
// exchange of the new ghost layers on the side stream while the persistent
// kernel steps the remaining nodes; walls and the finalise after both.
// second stream and the fork/join events of the step graphs (created once)
cudaError_t ensure_side(cavity *h) {
  cudaError_t e = cudaSuccess;
  if (!h->side) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && !h->ev_shell) e = cudaEventCreateWithFlags(&h->ev_shell, cudaEventDisableTiming);
  if (e == cudaSuccess && !h->ev_exch) e = cudaEventCreateWithFlags(&h->ev_exch, cudaEventDisableTiming);
  return e;
}

int launch_step_overlapped(cavity *h, int parity) {
  const ShellArgs sa{h->d_blocks, h->d_shell, (int)h->hshell.size(), h->d_cc, h->d_cs, h->d_step_part,
                     (long long)h->n_step, parity, h->local_dt};
  k_shell_f64<<<h->n_shell, kShellThreads, 0, h->stream>>>(sa);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev_shell, h->stream));
  CK(cudaStreamWaitEvent(h->side, h->ev_shell, 0));
  launch_pack(h, parity ^ 1, h->side);
  launch_unpack(h, parity ^ 1, h->side);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev_exch, h->side));
  StepArgs st = step_args(h, parity, 0);
  st.skip_shell = 1;
  launch_step_f64(h, st);
  CK(cudaGetLastError());
  CK(cudaStreamWaitEvent(h->stream, h->ev_exch, 0));
  // the finalise with the walls (and their Nusselt partials) in the same launch
  BcArgs ba = bc_args(h, parity ^ 1, 0);
  ba.wall_ctas = h->n_bc;
  ba.shell_begin = h->n_step;
  ba.shell_end = (long long)h->n_step + h->n_shell;
  k_finalize<double><<<h->ncav * h->nslices + h->n_bc, kFinThreads, 0, h->stream>>>(ba, h->d_fin);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// one explicit step reading buffer set `parity`, leaving the new state in parity ^ 1
// (the exchange of a decomposed cavity runs inside the finalise launch)
int launch_step(cavity *h, int parity, bool after_finalise = false) {
  if (h->overlap) return launch_step_overlapped(h, parity);
  launch_step_kernel(h, parity, after_finalise);
  CK(cudaGetLastError());
  launch_bc_kernel(h, parity ^ 1, 0);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// walls, ghosts, dt and Nusselt of the state in the current buffer set (no step)
int refresh_state(cavity *h) {
  launch_spectral(h);
  CK(cudaGetLastError());
  launch_bc_kernel(h, h->parity, 1);
  CK(cudaGetLastError());
  return launch_exchange(h, h->parity);
}

void drop_graphs(cavity *h) {
  for (auto &g : h->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (auto &g : h->graph2)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int build_graphs(cavity *h) {
  drop_graphs(h);
  if (h->n_cut > 0) CK(ensure_side(h));
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
  for (int par = 0; par < 2; ++par) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_step(h, par);
    if (rc == CAVITY_OK) rc = launch_step(h, par ^ 1, true);
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != CAVITY_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e);
    const cudaError_t e2 = cudaGraphInstantiate(&h->graph2[par], g, 0);
    cudaGraphDestroy(g);
    CK(e2);
  }
  return CAVITY_OK;
}

// change the FP32 step kernel's tile shape: work lists, maps, graphs
int retile(cavity *h, int p, int ty, int kc, int r) {
  CK(cudaStreamSynchronize(h->stream));
  h->f32_p = p;
  h->ty = ty;
  h->kc = kc;
  h->f32_r = r;
  assign_tiles(h);
  int rc = ensure_partials(h);
  if (rc == CAVITY_OK) rc = upload_tables(h);
  if (rc == CAVITY_OK) rc = encode_maps(h);
  if (rc != CAVITY_OK) return rc;
  CK(f32_set_smem(p, ty, r));
  return build_graphs(h);
}

int init_state(cavity *h) {
  CK(cudaMemsetAsync(h->d_fields, 0, h->field_bytes, h->stream));
  CK(cudaMemsetAsync(h->d_cs, 0, sizeof(CavState) * h->ncav, h->stream));
  h->parity = 0;
  h->steps_taken = 0;
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    const cavity_desc &d = h->descs[B.cav];
    const cavity_params &p = h->prms[B.cav];
    InitArgs a{h->d_blocks, h->d_cc, id, 0, d.seed, d.noise_amp, p.t_hot, p.t_cold};
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

int read_states(cavity *h, std::vector<CavState> &st) {
  st.resize(h->ncav);
  CK(cudaMemcpyAsync(st.data(), h->d_cs, sizeof(CavState) * h->ncav, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int read_state(cavity *h, int cav, CavState *st) {
  CK(cudaMemcpyAsync(st, h->d_cs + cav, sizeof(CavState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int state_status(const CavState &st) {
  if (st.flags & 2) return CAVITY_ERR_TIMEOUT;
  if (st.flags & 1) return CAVITY_ERR_NONFINITE;
  return CAVITY_OK;
}

int all_status(cavity *h) {
  std::vector<CavState> st;
  int rc = read_states(h, st);
  if (rc != CAVITY_OK) return rc;
  int worst = CAVITY_OK;
  for (const CavState &s : st) {
    const int r = state_status(s);
    if (r == CAVITY_ERR_TIMEOUT) return r;
    if (r != CAVITY_OK) worst = r;
  }
  return worst;
}

int get_fields_cav(cavity *h, int cav, int mask, double *host, size_t count) {
  if (!host || mask <= 0 || mask > CAVITY_FIELD_ALL || cav < 0 || cav >= h->ncav) return CAVITY_ERR_INVALID_ARG;
  const cavity_desc &d = h->descs[cav];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  if (count != (size_t)popcount5(mask) * N) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, cav, &st);
  if (rc != CAVITY_OK) return rc;
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    if (B.cav != cav) continue;
    MoveArgs a{h->d_blocks, id, h->parity, mask, {d.nx, d.ny, d.nz}, h->d_stage, st.c};
    const int grid = ceil_div((long long)B.nx * B.ny * B.nz, 256);
    if (h->f32) k_gather<float><<<grid, 256, 0, h->stream>>>(a);
    else k_gather<double><<<grid, 256, 0, h->stream>>>(a);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(host, h->d_stage, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

void release(cavity *h) {
  DeviceGuard g(h->dev);
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  void *ptrs[] = {h->d_fields, h->d_blocks, h->d_cc, h->d_cs, h->d_wall, h->d_cut, h->d_step_part,
                  h->d_bc_part, h->d_counter, h->d_twall, h->d_xbuf, h->d_stage, h->d_maps, h->d_fin, h->d_shell};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  AdjointStore &A = h->adj;
  void *aptrs[] = {A.ckpt_mem, A.ckpt_cs, A.seg_mem, A.final_mem, A.X, A.Yt, A.Q, A.thetabar, A.scal,
                   A.argpart, A.gpart, A.dts, A.block, A.seg_blocks, A.seg_faces, A.seg_maps, A.cnt};
  for (void *p : aptrs)
    if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_shell) cudaEventDestroy(h->ev_shell);
  if (h->ev_exch) cudaEventDestroy(h->ev_exch);
  for (cudaEvent_t e : h->adj_ev) cudaEventDestroy(e);
  h->adj_ev.clear();
}

int create_common(const cavity_desc *descs, const cavity_params *params, int n, cavity_t **out) {
  if (!out) return CAVITY_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n < 1) return CAVITY_ERR_INVALID_ARG;
  for (int c = 0; c < n; ++c) {
    if (check_desc(descs[c]) != CAVITY_OK) return CAVITY_ERR_INVALID_ARG;
    if (n > 1 && (descs[c].px != 1 || descs[c].py != 1 || descs[c].pz != 1)) return CAVITY_ERR_INVALID_ARG;
    if (descs[c].precision != descs[0].precision) return CAVITY_ERR_INVALID_ARG;
    if (params) {
      cavity_params q = params[c];
      resolve_defaults(&q);
      if (check_params(q) != CAVITY_OK) return CAVITY_ERR_INVALID_ARG;
    }
  }
  const cavity_desc &d0 = descs[0];
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d0.device < 0 || d0.device >= ndev) return CAVITY_ERR_CUDA;
  cavity *h = new (std::nothrow) cavity();
  if (!h) return CAVITY_ERR_OOM;
  h->ncav = n;
  h->descs.assign(descs, descs + n);
  h->prms.resize(n);
  for (int c = 0; c < n; ++c) {
    if (params) {
      h->prms[c] = params[c];
      resolve_defaults(&h->prms[c]);
    } else {
      cavity_default_params(&h->prms[c]);
    }
  }
  h->hcc.assign(n, CavConst{});
  h->wall_custom.assign(2 * n, 0);
  h->dev = d0.device;
  h->f32 = d0.precision == CAVITY_FP32_MIXED;
  h->esize = h->f32 ? 4 : 8;
  h->na = h->f32 ? Store<float>::NA : Store<double>::NA;
  h->np = h->f32 ? Store<float>::NP : Store<double>::NP;
  if (!h->f32) {
    // tile-height override for tuning sweeps: BDC_F64_TY=4 or 8
    if (const char *env = std::getenv("BDC_F64_TY")) {
      const int ty = std::atoi(env);
      if (ty == 4 || ty == 8) h->ty = ty;
    }
  }
  if (h->f32) {
    h->tx = kF32TX;
    h->ty = kF32TY;
    h->kc = kF32KC;
    h->f32_r = kF32R;
    h->f32_p = 3;
    // shape override for tuning sweeps: BDC_F32_TILE="TY,KC,R[,P]" (a compiled shape)
    if (const char *env = std::getenv("BDC_F32_TILE")) {
      int ty = 0, kc = 0, r = 0, p = 3;
      const int got = std::sscanf(env, "%d,%d,%d,%d", &ty, &kc, &r, &p);
      if (got >= 3 && f32_variant_ok(p, ty, kc, r)) {
        h->ty = ty;
        h->kc = kc;
        h->f32_r = r;
        h->f32_p = p;
      }
    }
  }
  int rc = CAVITY_OK;
  {
    DeviceGuard g(h->dev);
    if (d0.stream) {
      h->stream = (cudaStream_t)d0.stream;
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

}  // namespace

// ===========================================================================
// the reverse of one step: state storage S, adjoint arrays and arithmetic Ad
template <class S, class Ad>
void launch_adjoint_step(cavity *h, const AdjArgs &a, int nparts, long long nint, long long nfold, cudaEvent_t eb,
                         cudaEvent_t ea) {
  if constexpr (std::is_same<Ad, float>::value) {
    // FP32 sweep: the objective, the p-adjoint sum and the centre-shift
    // transpose in place on X in one launch, then the gather reads X as Yt
    // (no atomics, no full prepare pass); the argmax of this state came with
    // its segment's (a.argpart), and the dt kernel reduces the gather's
    // partials itself
    k_adj_pre<Ad><<<nparts, 256, 0, h->stream>>>(a, h->adj.cnt);
    AdjArgs g = a;
    g.Yt = a.X;
    cudaEventRecord(eb, h->stream);
    k_adj_gather<<<ceil_div(a.g.fs, 256), 256, 0, h->stream>>>(g);
    cudaEventRecord(ea, h->stream);
    AdjArgs d = a;
    d.gpart2 = nullptr;
    k_adj_dt<S, Ad><<<1, kAdjDtThreads, 0, h->stream>>>(d, nparts);
  } else {
    k_adj_objective<Ad><<<ceil_div((long long)a.g.ny * a.g.nz, 256), 256, 0, h->stream>>>(a);
    k_adj_sum_p<Ad><<<nparts, 256, 0, h->stream>>>(a);
    k_adj_prepare<Ad, true><<<dim3((unsigned)ceil_div(a.g.fs, 256), 5), 256, 0, h->stream>>>(a);
    cudaEventRecord(eb, h->stream);
    k_adj_rates<S, Ad><<<ceil_div(nint, 256), 256, 0, h->stream>>>(a);
    cudaEventRecord(ea, h->stream);
    k_adj_argmax<S><<<nparts, 256, 0, h->stream>>>(a);
    k_adj_dt<S, Ad><<<1, kAdjDtThreads, 0, h->stream>>>(a, nparts);
  }
  k_adj_fold<Ad><<<ceil_div(nfold, 256), 256, 0, h->stream>>>(a);
}

// cavity_check_sqrt: relative difference of sqrt_newton from CUDA's sqrt
__global__ void k_check_sqrt(const double *x, long long n, double *rel) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = sqrt(x[i]), s = sqrt_newton(x[i]);
  rel[i] = s == r ? 0.0 : fabs(s - r) / r;
}

// cavity_check_div3: whether div3 equals CUDA's correctly rounded x / 3
__global__ void k_check_div3(const double *x, long long n, unsigned char *diff) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  diff[i] = div3(x[i]) != x[i] / 3.0;
}

// Recomputation of a checkpointed segment without copies: points block 0 of
// the step graph's descriptor table at two buffer sets -- base[0] (read) = b0,
// base[1] (written) = b1 -- and, in the FP32 form, replaces the parity-0
// tensor maps with b0's (src[0], src[1]), so the captured one-step graph of
// parity 0 steps the state in slot s straight into slot s + 1.  One warp.
__global__ void k_adj_point(BlockDev *blk, CUtensorMap *maps, const CUtensorMap *src, void *b0, void *b1) {
  if (threadIdx.x == 0) {
    blk->base[0] = b0;
    blk->base[1] = b1;
  }
  if (maps) {
    static_assert(sizeof(CUtensorMap) == 128, "two 128-byte maps, 8 bytes per lane");
    reinterpret_cast<unsigned long long *>(maps)[threadIdx.x] =
        reinterpret_cast<const unsigned long long *>(src)[threadIdx.x];
    // the maps are read through the tensor-map proxy by the next kernel
    asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
  }
}

// FP64 FMA throughput of the GPU: every thread runs kDfmaChains independent
// chains x <- x a + b (a = 1 - 2^-20, b = 2^-20: the values stay near 1, no
// overflow or subnormals), unrolled so that the FP64 pipe always has an
// independent FMA to issue; the sum is compared with a value it never takes,
// so no chain can be removed.  FLOPs = 2 per FMA.
constexpr int kDfmaChains = 8, kDfmaUnroll = 4, kDfmaThreads = 256;
__global__ void __launch_bounds__(kDfmaThreads) k_dfma_peak(double *sink, int iters, double a, double b) {
  double x[kDfmaChains];
#pragma unroll
  for (int c = 0; c < kDfmaChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kDfmaUnroll; ++r)
#pragma unroll
      for (int c = 0; c < kDfmaChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kDfmaChains; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

extern "C" {

int cavity_default_params(cavity_params *p) {
  if (!p) return CAVITY_ERR_INVALID_ARG;
  p->Ra = 1e5; p->Pr = 0.71; p->cfl = 0.5; p->kappa = 0.1; p->c4 = 1.0 / 32.0;
  p->u_ref = -1.0; p->t_inf = NAN; p->t_hot = 1.0; p->t_cold = 0.0; p->gravity_axis = 2;
  resolve_defaults(p);
  return CAVITY_OK;
}

int cavity_create(const cavity_desc *desc, cavity_t **out) { return create_common(desc, nullptr, 1, out); }

int cavity_create_batch(const cavity_desc *descs, const cavity_params *params, int n, cavity_t **out) {
  return create_common(descs, params, n, out);
}

int cavity_batch_size(cavity_t *h) { return h ? h->ncav : CAVITY_ERR_INVALID_ARG; }

int cavity_set_params(cavity_t *h, const cavity_params *p) {
  if (!h || !p) return CAVITY_ERR_INVALID_ARG;
  cavity_params q = *p;
  const bool auto_uref = !(q.u_ref >= 0.0);
  resolve_defaults(&q);
  if (check_params(q) != CAVITY_OK) return fail(h, CAVITY_ERR_INVALID_ARG, "invalid parameters");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  h->u_ref_auto = auto_uref;
  for (auto &pc : h->prms) pc = q;
  int rc = upload_consts(h);
  if (rc != CAVITY_OK) return rc;
  if (h->steps_taken == 0) return init_state(h);
  return refresh_state(h);
}

int cavity_set_wall_temperature(cavity_t *h, int wall, const double *host, size_t n) {
  if (!h || !host || (wall != 0 && wall != 1)) return CAVITY_ERR_INVALID_ARG;
  const size_t nw = (size_t)h->descs[0].ny * h->descs[0].nz;
  if (n != nw) return fail(h, CAVITY_ERR_INVALID_ARG, "wall temperature count must be ny*nz");
  for (size_t q = 0; q < n; ++q)
    if (!std::isfinite(host[q])) return fail(h, CAVITY_ERR_INVALID_ARG, "non-finite wall temperature");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  std::copy(host, host + n, h->twall.begin() + h->hcc[0].wall_off + (wall ? nw : 0));
  h->wall_custom[wall] = 1;
  int rc = upload_consts(h);
  if (rc != CAVITY_OK) return rc;
  return refresh_state(h);
}

int cavity_step(cavity_t *h, int nsteps) {
  if (!h || nsteps < 0) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  int s = 0;
  for (; s + 2 <= nsteps; s += 2) {  // two steps per graph: the parity comes back
    CK(cudaGraphLaunch(h->graph2[h->parity], h->stream));
    h->steps_taken += 2;
  }
  if (s < nsteps) {
    CK(cudaGraphLaunch(h->graph[h->parity], h->stream));
    h->parity ^= 1;
    h->steps_taken += 1;
  }
  return CAVITY_OK;
}

int cavity_batch_state(cavity_t *h, int cav, double out[10]) {
  if (!h || !out || cav < 0 || cav >= h->ncav) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, cav, &st);
  if (rc != CAVITY_OK) return rc;
  out[0] = (double)st.step;
  out[1] = st.t;
  out[2] = st.dt;
  for (int f = 0; f < 5; ++f) out[3 + f] = st.res[f];
  out[8] = st.nu_hot;
  out[9] = st.nu_cold;
  return state_status(st);
}

int cavity_batch_get_fields(cavity_t *h, int cav, int mask, double *host, size_t count) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  return get_fields_cav(h, cav, mask, host, count);
}

static_assert(sizeof(StepRecord) == sizeof(cavity_step_record), "step record layout");
static_assert(offsetof(StepRecord, flags) == offsetof(cavity_step_record, flags), "step record layout");

int cavity_set_step_log(cavity_t *h, cavity_step_record *host, long long capacity) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  StepRecord *dev = nullptr;
  if (host) {
    if (capacity < 1) return fail(h, CAVITY_ERR_INVALID_ARG, "step log: capacity < 1");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, host) != cudaSuccess || pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
      cudaGetLastError();
      return fail(h, CAVITY_ERR_INVALID_ARG, "step log: not page-locked host memory the device can address");
    }
    dev = (StepRecord *)pa.devicePointer;
  }
  CK(cudaStreamSynchronize(h->stream));
  h->d_log = dev;
  h->log_cap = host ? capacity : 0;
  return build_graphs(h);  // the finalise launches in the graphs carry the log
}

int cavity_step_log_alloc(long long records, cavity_step_record **out) {
  if (!out || records < 1 || records > (1LL << 32)) return CAVITY_ERR_INVALID_ARG;
  *out = nullptr;
  void *p = nullptr;
  const size_t bytes = (size_t)records * sizeof(cavity_step_record);
  if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    return CAVITY_ERR_OOM;
  }
  std::memset(p, 0, bytes);
  *out = (cavity_step_record *)p;
  return CAVITY_OK;
}

int cavity_step_log_free(cavity_step_record *p) {
  if (p && cudaFreeHost(p) != cudaSuccess) return CAVITY_ERR_CUDA;
  return CAVITY_OK;
}

int cavity_residual(cavity_t *h, double out[5]) {
  if (!h || !out) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, 0, &st);
  if (rc != CAVITY_OK) return rc;
  for (int f = 0; f < 5; ++f) out[f] = st.res[f];
  return state_status(st);
}

int cavity_nusselt(cavity_t *h, double *hot, double *cold) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, 0, &st);
  if (rc != CAVITY_OK) return rc;
  if (hot) *hot = st.nu_hot;
  if (cold) *cold = st.nu_cold;
  return state_status(st);
}

int cavity_get_time(cavity_t *h, long long *step, double *t, double *dt) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CavState st;
  int rc = read_state(h, 0, &st);
  if (rc != CAVITY_OK) return rc;
  if (step) *step = st.step;
  if (t) *t = st.t;
  if (dt) *dt = st.dt;
  return state_status(st);
}

int cavity_get_fields(cavity_t *h, int mask, double *host, size_t count) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  return get_fields_cav(h, 0, mask, host, count);
}

int cavity_get_fields_box(cavity_t *h, int mask, int i0, int j0, int k0, int ni, int nj, int nk, double *host,
                          size_t count) {
  if (!h || !host || mask <= 0 || mask > CAVITY_FIELD_ALL) return CAVITY_ERR_INVALID_ARG;
  const cavity_desc &d = h->descs[0];
  if (ni < 1 || nj < 1 || nk < 1 || i0 < 1 || j0 < 1 || k0 < 1 || i0 + ni - 1 > d.nx || j0 + nj - 1 > d.ny ||
      k0 + nk - 1 > d.nz)
    return fail(h, CAVITY_ERR_INVALID_ARG, "box outside the interior");
  const size_t n = (size_t)ni * nj * nk;
  if (count != (size_t)popcount5(mask) * n) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, 0, &st);
  if (rc != CAVITY_OK) return rc;
  int nb0 = 0;  // blocks of cavity 0
  while (nb0 < h->nblocks && h->hb[nb0].cav == 0) ++nb0;
  BoxArgs a{h->d_blocks, nb0, h->parity, mask, i0, j0, k0, ni, nj, nk, h->d_stage, st.c};
  if (h->f32) k_gather_box<float><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(a);
  else k_gather_box<double><<<ceil_div((long long)n, 256), 256, 0, h->stream>>>(a);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host, h->d_stage, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAVITY_OK;
}

int cavity_set_fields(cavity_t *h, int mask, const double *host, size_t count) {
  if (!h || !host || mask <= 0 || mask > CAVITY_FIELD_ALL) return CAVITY_ERR_INVALID_ARG;
  const cavity_desc &d = h->descs[0];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  if (count != (size_t)popcount5(mask) * N) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
  DeviceGuard g(h->dev);
  int rc = ensure_stage(h, count);
  if (rc != CAVITY_OK) return rc;
  CavState st;
  rc = read_state(h, 0, &st);
  if (rc != CAVITY_OK) return rc;
  // fold the pending centre shift into the stored p, then c = 0
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    if (B.cav != 0) continue;
    if (st.c != 0.0 && !(mask & CAVITY_FIELD_P)) {
      const int grid = ceil_div((long long)(B.nx + 4) * (B.ny + 4) * (B.nz + 4), 256);
      if (h->f32) k_shift_p<float><<<grid, 256, 0, h->stream>>>(h->d_blocks, id, h->parity, st.c);
      else k_shift_p<double><<<grid, 256, 0, h->stream>>>(h->d_blocks, id, h->parity, st.c);
      CK(cudaGetLastError());
    }
  }
  CK(cudaMemsetAsync(&h->d_cs[0].c, 0, sizeof(double), h->stream));
  CK(cudaMemcpyAsync(h->d_stage, host, count * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  for (int id = 0; id < h->nblocks; ++id) {
    const BlockDev &B = h->hb[id];
    if (B.cav != 0) continue;
    MoveArgs a{h->d_blocks, id, h->parity, mask, {d.nx, d.ny, d.nz}, h->d_stage, 0.0};
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
    const size_t n = (size_t)(h->na + h->np) * c.nb * c.nc;
    if (count != n) return fail(h, CAVITY_ERR_INVALID_ARG, "count mismatch");
    DeviceGuard g(h->dev);
    // the step's exchange writes the ghost layers directly: pack the current
    // state's faces (the values every exchange of this state sends)
    launch_pack(h, h->parity);
    CK(cudaGetLastError());
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

int cavity_autotune(cavity_t *h, int steps, double out[5]) {
  if (!h || steps < 1) return CAVITY_ERR_INVALID_ARG;
  if (!h->f32) return fail(h, CAVITY_ERR_UNSUPPORTED, "the FP64 form has one tile shape");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  if (std::getenv("BDC_F32_TILE")) {  // a pinned shape (set at creation): no trials
    if (out) {
      out[0] = h->ty;
      out[1] = h->kc;
      out[2] = h->f32_r;
      out[3] = h->f32_p;
      out[4] = 0.0;
    }
    return CAVITY_OK;
  }
  // save the state (fields, per-cavity scalars, ping-pong parity, step count)
  void *backup = nullptr;
  CK(cudaMalloc(&backup, h->field_bytes));
  std::vector<CavState> st0;
  int rc = read_states(h, st0);
  const int par0 = h->parity;
  const long long steps0 = h->steps_taken;
  auto restore = [&]() -> int {
    CK(cudaMemcpyAsync(h->d_fields, backup, h->field_bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_cs, st0.data(), sizeof(CavState) * h->ncav, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->parity = par0;
    h->steps_taken = steps0;
    return CAVITY_OK;
  };
  if (rc == CAVITY_OK && cudaMemcpyAsync(backup, h->d_fields, h->field_bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    rc = fail(h, CAVITY_ERR_CUDA, "state backup failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == CAVITY_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(h, CAVITY_ERR_CUDA, "event creation failed");
  // one trial of a shape: `steps` graph-replayed steps after a warm-up, from the saved state
  auto trial = [&](const F32Shape &s, double &us) -> int {
    int r = retile(h, s.p, s.ty, s.kc, s.r);
    if (r == CAVITY_OK) r = cavity_step(h, 2);  // warm-up
    if (r != CAVITY_OK) return r;
    cudaEventRecord(e0, h->stream);
    r = cavity_step(h, steps);
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) r = fail(h, CAVITY_ERR_CUDA, "trial failed");
    if (r != CAVITY_OK) return r;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    us = 1e3 * ms / steps;
    return restore();
  };
  // every shape once, then the four fastest again (each keeps its better
  // time): one trial's noise between close shapes no longer decides
  const std::vector<F32Shape> shapes = f32_shapes();
  std::vector<double> t(shapes.size(), 1e300);
  for (size_t q = 0; q < shapes.size() && rc == CAVITY_OK; ++q) rc = trial(shapes[q], t[q]);
  std::vector<size_t> order(shapes.size());
  for (size_t q = 0; q < order.size(); ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return t[x] < t[y]; });
  for (size_t q = 0; q < std::min<size_t>(4, order.size()) && rc == CAVITY_OK; ++q) {
    double us = 1e300;
    rc = trial(shapes[order[q]], us);
    t[order[q]] = std::min(t[order[q]], us);
  }
  double best_us = 1e300;
  F32Shape best = {h->f32_p, h->ty, h->kc, h->f32_r};
  for (size_t q = 0; q < shapes.size(); ++q)
    if (t[q] < best_us) {
      best_us = t[q];
      best = shapes[q];
    }
  if (rc == CAVITY_OK) rc = retile(h, best.p, best.ty, best.kc, best.r);
  if (rc == CAVITY_OK) rc = restore();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(backup);
  if (rc == CAVITY_OK && out) {
    out[0] = best.ty;
    out[1] = best.kc;
    out[2] = best.r;
    out[3] = best.p;
    out[4] = best_us;
  }
  return rc;
}

int cavity_adjoint_forward(cavity_t *h, int nsteps, int ckpt, double *J) {
  if (!h || nsteps < 1 || ckpt < 1) return CAVITY_ERR_INVALID_ARG;
  if (h->local_dt) return fail(h, CAVITY_ERR_UNSUPPORTED, "adjoint: global time stepping only");
  if ((long long)(h->descs[0].nx + 4) * (h->descs[0].ny + 4) * (h->descs[0].nz + 4) >= (1LL << 31))
    return fail(h, CAVITY_ERR_UNSUPPORTED, "adjoint: fewer than 2^31 nodes with the two-node halo");
  if (h->ncav != 1 || h->nblocks != 1) return fail(h, CAVITY_ERR_UNSUPPORTED, "adjoint: single-block cavity only");
  DeviceGuard g(h->dev);
  AdjointStore &A = h->adj;
  const BlockDev &B = h->hb[0];
  const cavity_desc &d = h->descs[0];
  const size_t set_bytes = (size_t)h->na * (size_t)B.fstride * h->esize;
  const int ncp = (nsteps + ckpt - 1) / ckpt;
  const long long fs = (long long)(d.nx + 4) * (d.ny + 4) * (d.nz + 4);
  const int nparts = 2 * 152;
  CK(cudaStreamSynchronize(h->stream));
  if (A.set_bytes != set_bytes || A.ncp < ncp || A.ckpt < ckpt || A.nsteps < nsteps) {
    void *aptrs[] = {A.ckpt_mem, A.ckpt_cs, A.seg_mem, A.final_mem, A.X, A.Yt, A.Q, A.thetabar, A.scal,
                     A.argpart, A.gpart, A.dts, A.block, A.seg_blocks, A.seg_faces, A.seg_maps, A.cnt};
    for (void *p : aptrs)
      if (p) cudaFree(p);
    A = AdjointStore{};
    CK(cudaMalloc(&A.ckpt_mem, set_bytes * ncp));
    CK(cudaMalloc(&A.ckpt_cs, sizeof(CavState) * ncp));
    CK(cudaMalloc(&A.seg_mem, set_bytes * ckpt));
    CK(cudaMalloc(&A.final_mem, set_bytes));
    const size_t abytes = (h->f32 ? sizeof(float) : sizeof(double)) * 5 * fs;
    CK(cudaMalloc(&A.X, abytes));
    CK(cudaMalloc(&A.Yt, abytes));
    CK(cudaMalloc(&A.Q, abytes));
    CK(cudaMalloc(&A.thetabar, sizeof(double) * d.ny * d.nz));
    CK(cudaMalloc(&A.scal, sizeof(double) * kScCount));
    CK(cudaMalloc(&A.argpart, sizeof(double) * 2 * nparts * ckpt));  // one set per segment slot
    CK(cudaMalloc(&A.cnt, sizeof(unsigned int)));
    CK(cudaMemset(A.cnt, 0, sizeof(unsigned int)));
    CK(cudaMalloc(&A.gpart, sizeof(double) * 3 * (ceil_div(fs, 256) + nparts)));
    CK(cudaMalloc(&A.dts, sizeof(double) * nsteps));
    CK(cudaMalloc(&A.block, sizeof(BlockDev)));
    A.set_bytes = set_bytes;
    // per segment slot: its block descriptor, its wall faces (one walls
    // launch covers the segment) and, in the FP32 form, its tensor maps
    std::vector<BlockDev> sb(ckpt, h->hb[0]);
    std::vector<WallFace> sf;
    for (int s = 0; s < ckpt; ++s) {
      sb[s].base[0] = A.seg_mem + (size_t)s * set_bytes;
      for (WallFace f : h->hwall) {
        f.block = s;
        f.cta_begin += s * h->n_bc;
        sf.push_back(f);
      }
    }
    CK(cudaMalloc(&A.seg_blocks, sizeof(BlockDev) * ckpt));
    CK(cudaMalloc(&A.seg_faces, sizeof(WallFace) * sf.size()));
    CK(cudaMemcpy(A.seg_blocks, sb.data(), sizeof(BlockDev) * ckpt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(A.seg_faces, sf.data(), sizeof(WallFace) * sf.size(), cudaMemcpyHostToDevice));
    if (h->f32) {
      std::vector<CUtensorMap> sm(2 * (size_t)ckpt);
      for (int s = 0; s < ckpt; ++s) {
        const int rc = encode_block_maps(h, h->hb[0], A.seg_mem + (size_t)s * set_bytes, &sm[2 * s]);
        if (rc != CAVITY_OK) return rc;
      }
      CK(cudaMalloc(&A.seg_maps, sizeof(CUtensorMap) * sm.size()));
      CK(cudaMemcpy(A.seg_maps, sm.data(), sizeof(CUtensorMap) * sm.size(), cudaMemcpyHostToDevice));
    }
  }
  A.nsteps = nsteps;
  A.ckpt = ckpt;
  A.ncp = ncp;
  A.nparts = nparts;
  // every segment slot starts as a copy of the initial state: the step
  // writes interior nodes and the walls that change (p, adiabatic T), so the
  // constant wall values (u = v = w = 0, the isothermal T) a recomputed state
  // is read with must already be in its slot
  for (int s = 0; s < ckpt; ++s)
    CK(cudaMemcpyAsync(A.seg_mem + (size_t)s * set_bytes, h->hb[0].base[h->parity], set_bytes,
                       cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemsetAsync(A.scal, 0, sizeof(double) * kScCount, h->stream));
  for (int n = 0; n < nsteps; ++n) {
    if (n % ckpt == 0) {
      const int c = n / ckpt;
      CK(cudaMemcpyAsync(A.ckpt_mem + (size_t)c * set_bytes, h->hb[0].base[h->parity], set_bytes,
                         cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(A.ckpt_cs + c, h->d_cs, sizeof(CavState), cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(cudaGraphLaunch(h->graph[h->parity], h->stream));
    h->parity ^= 1;
    h->steps_taken += 1;
    k_adj_acc_nusselt<<<1, 1, 0, h->stream>>>(h->d_cs, A.scal);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(A.final_mem, h->hb[0].base[h->parity], set_bytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(&A.final_cs, h->d_cs, sizeof(CavState), cudaMemcpyDeviceToHost, h->stream));
  double acc = 0.0;
  CK(cudaMemcpyAsync(&acc, A.scal + kScJ, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  A.final_parity = h->parity;
  A.final_steps = h->steps_taken;
  A.J = acc / nsteps;
  A.have_forward = true;
  if (J) *J = A.J;
  return state_status(A.final_cs);
}

int cavity_adjoint_backward(cavity_t *h, double *grad_wall, size_t n, double *grad_ra) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  AdjointStore &A = h->adj;
  if (!A.have_forward) return fail(h, CAVITY_ERR_INVALID_ARG, "adjoint: no forward run recorded");
  const cavity_desc &d = h->descs[0];
  if (grad_wall && n != (size_t)d.ny * d.nz) return fail(h, CAVITY_ERR_INVALID_ARG, "grad_wall count must be ny*nz");
  DeviceGuard g(h->dev);
  const BlockDev B0 = h->hb[0];
  const cavity_params &p = h->prms[0];
  AdjArgs a{};
  a.C = h->hcc[0];
  a.g = AdjGeom{d.nx, d.ny, d.nz, (long long)d.nx + 4, (long long)d.ny + 4,
                (long long)(d.nx + 4) * (d.ny + 4) * (d.nz + 4)};
  a.Yt = A.Yt;
  a.scal = A.scal;
  a.thetabar = A.thetabar;
  a.argpart = A.argpart;
  a.gpart = A.gpart;
  a.ngpart = h->f32 ? (int)ceil_div(a.g.fs, 256) : 0;
  a.gpart2 = A.gpart + 3 * ceil_div(a.g.fs, 256);
  a.coef = 1.0 / ((double)A.nsteps * d.ny * d.nz * 2.0 * a.C.h[0] * (p.t_hot - p.t_cold));
  a.dfloor = (h->u_ref_auto && p.Ra * p.Pr > 1.0) ? p.kappa * p.Pr : 0.0;
  void *X = A.X, *Q = A.Q;
  CK(cudaMemsetAsync(X, 0, (h->f32 ? sizeof(float) : sizeof(double)) * 5 * a.g.fs, h->stream));
  CK(cudaMemsetAsync(A.thetabar, 0, sizeof(double) * d.ny * d.nz, h->stream));
  CK(cudaMemsetAsync(A.scal, 0, sizeof(double) * kScCount, h->stream));
  const long long nint = (long long)d.nx * d.ny * d.nz;
  const long long nfold = 2LL * ((long long)d.ny * d.nz + (long long)d.nx * d.nz + (long long)d.nx * d.ny);
  std::vector<double> dts(A.ckpt);
  while (h->adj_ev.size() < 2 * (size_t)A.nsteps) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreate(&e));
    h->adj_ev.push_back(e);
  }
  int rc = CAVITY_OK;
  auto slot = [&](int s) { return (void *)(A.seg_mem + (size_t)s * A.set_bytes); };
  for (int c = A.ncp - 1; c >= 0 && rc == CAVITY_OK; --c) {
    const int s0 = c * A.ckpt, s1 = std::min(s0 + A.ckpt, A.nsteps);
    // recompute the segment from its checkpoint (copied to slot 0), each step
    // of the parity-0 graph reading slot s - s0 and writing slot s - s0 + 1
    CK(cudaMemcpyAsync(slot(0), A.ckpt_mem + (size_t)c * A.set_bytes, A.set_bytes, cudaMemcpyDeviceToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(h->d_cs, A.ckpt_cs + c, sizeof(CavState), cudaMemcpyDeviceToDevice, h->stream));
    for (int s = s0; s < s1; ++s) {
      CK(cudaMemcpyAsync(A.dts + s, &h->d_cs->dt, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      if (s < s1 - 1) {
        k_adj_point<<<1, 32, 0, h->stream>>>(h->d_blocks, h->f32 ? h->d_maps : nullptr,
                                             h->f32 ? A.seg_maps + 2 * (s - s0) : nullptr, slot(s - s0),
                                             slot(s - s0 + 1));
        CK(cudaGetLastError());
        CK(cudaGraphLaunch(h->graph[0], h->stream));
      }
    }
    if (h->f32) {
      // the FP32-mixed step forms p's and T's wall values where it reads
      // them: write them into every stored state of the segment, one launch
      BcArgs ba = bc_args(h, 0, 3);
      ba.blocks = A.seg_blocks;
      ba.faces = A.seg_faces;
      ba.nfaces = (int)h->hwall.size() * (s1 - s0);
      ba.tile_counter = nullptr;
      ba.sfloor = nullptr;
      k_bc<float><<<h->n_bc * (s1 - s0), kBcThreads, 0, h->stream>>>(ba);
      CK(cudaGetLastError());
      // the argmax of every state of the segment's spectral bound, one launch
      k_adj_argmax_seg<float><<<dim3(A.nparts, s1 - s0), 256, 0, h->stream>>>(A.seg_blocks, h->hcc[0], a.g, A.argpart);
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(dts.data(), A.dts + s0, sizeof(double) * (s1 - s0), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // reverse sweep over the segment
    for (int s = s1 - 1; s >= s0; --s) {
      a.B = B0;
      a.B.base[0] = slot(s - s0);
      a.dt = dts[s - s0];
      a.argpart = h->f32 ? A.argpart + 2 * (size_t)A.nparts * (s - s0) : A.argpart;
      a.X = X;
      a.Q = Q;
      cudaEvent_t eb = h->adj_ev[2 * s], ea = h->adj_ev[2 * s + 1];
      if (h->f32) launch_adjoint_step<float, float>(h, a, A.nparts, nint, nfold, eb, ea);
      else launch_adjoint_step<double, double>(h, a, A.nparts, nint, nfold, eb, ea);
      if (cudaGetLastError() != cudaSuccess) { rc = fail(h, CAVITY_ERR_CUDA, "adjoint kernel launch failed"); break; }
      std::swap(X, Q);
    }
  }
  // the step graph's table and maps back to the handle's buffers, and the
  // state after the forward run
  {
    const int r2 = upload_tables(h);
    if (r2 != CAVITY_OK) return r2;
    if (h->f32) {
      const int r3 = encode_maps(h);
      if (r3 != CAVITY_OK) return r3;
    }
  }
  CK(cudaMemcpyAsync(h->hb[0].base[A.final_parity], A.final_mem, A.set_bytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_cs, &A.final_cs, sizeof(CavState), cudaMemcpyHostToDevice, h->stream));
  h->parity = A.final_parity;
  h->steps_taken = A.final_steps;
  double ra = 0.0;
  CK(cudaMemcpyAsync(&ra, A.scal + kScRa, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (grad_wall)
    CK(cudaMemcpyAsync(grad_wall, A.thetabar, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (grad_ra) *grad_ra = ra;
  if (rc == CAVITY_OK) {
    double tot = 0.0;
    for (int s = 0; s < A.nsteps; ++s) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->adj_ev[2 * s], h->adj_ev[2 * s + 1]));
      tot += ms;
    }
    h->adj_rates_ms = tot / A.nsteps;
  }
  return rc;
}

int cavity_adjoint_kernel_ms(cavity_t *h, double *ms) {
  if (!h || !ms) return CAVITY_ERR_INVALID_ARG;
  if (h->adj_rates_ms <= 0.0) return fail(h, CAVITY_ERR_INVALID_ARG, "adjoint: no reverse sweep timed yet");
  *ms = h->adj_rates_ms;
  return CAVITY_OK;
}

int cavity_set_overlap(cavity_t *h, int on) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  if (on && (h->f32 || h->ncav != 1))
    return fail(h, CAVITY_ERR_UNSUPPORTED, "overlap: FP64 single-cavity handles only");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  h->overlap = on && h->n_cut > 0;  // nothing to overlap without cut faces
  if (h->overlap && h->hshell.empty()) {
    int cta = 0;
    for (int id = 0; id < h->nblocks; ++id) {
      const BlockDev &B = h->hb[id];
      const int n[3] = {B.nx, B.ny, B.nz};
      for (int f = 0; f < 6; ++f) {
        if (B.wall[f]) continue;
        const int a = f / 2;
        const int n1 = n[a == 0 ? 1 : 0], n2 = n[a == 2 ? 1 : 2];
        h->hshell.push_back(ShellFace{id, f, n1, n2, cta});
        cta += ceil_div(2LL * n1 * n2, kShellThreads);
      }
    }
    h->n_shell = cta;
    CK(cudaMalloc(&h->d_shell, sizeof(ShellFace) * h->hshell.size()));
    CK(cudaMemcpy(h->d_shell, h->hshell.data(), sizeof(ShellFace) * h->hshell.size(), cudaMemcpyHostToDevice));
    CK(ensure_side(h));
  }
  const int rc = ensure_partials(h);
  if (rc != CAVITY_OK) return rc;
  return build_graphs(h);
}

int cavity_set_time_stepping(cavity_t *h, int mode) {
  if (!h || (mode != CAVITY_DT_GLOBAL && mode != CAVITY_DT_LOCAL)) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  h->local_dt = mode == CAVITY_DT_LOCAL;
  return build_graphs(h);  // the kernels' arguments are part of the captured graphs
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
    // (the exchange runs inside the finalise launch: nothing here)
    cudaEventRecord(ev[3], h->stream);
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
  ms[2] = ms[3] = 0.0;
  return rc;
}

int cavity_check_div3(const double *x, long long n, long long *n_diff) {
  if (!x || !n_diff || n < 1 || n > (1ll << 26)) return CAVITY_ERR_INVALID_ARG;
  for (long long i = 0; i < n; ++i)
    if (!(std::fabs(x[i]) >= 4.0 * DBL_MIN && std::fabs(x[i]) <= DBL_MAX)) return CAVITY_ERR_INVALID_ARG;
  double *d = nullptr;
  const size_t bytes = (size_t)n * sizeof(double);
  cudaError_t e = cudaMalloc(&d, bytes + (size_t)n);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CAVITY_ERR_OOM : CAVITY_ERR_CUDA;
  std::vector<unsigned char> diff((size_t)n);
  e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_check_div3<<<(unsigned)((n + 255) / 256), 256>>>(d, n, (unsigned char *)(d + n));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(diff.data(), d + n, (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return CAVITY_ERR_CUDA;
  long long nd = 0;
  for (unsigned char c : diff) nd += c != 0;
  *n_diff = nd;
  return CAVITY_OK;
}

int cavity_check_sqrt(const double *x, long long n, double *max_rel, long long *n_diff) {
  if (!x || !max_rel || !n_diff || n < 1 || n > (1ll << 26)) return CAVITY_ERR_INVALID_ARG;
  for (long long i = 0; i < n; ++i)
    if (!(x[i] >= DBL_MIN && x[i] <= DBL_MAX)) return CAVITY_ERR_INVALID_ARG;
  double *d = nullptr;
  const size_t bytes = (size_t)n * sizeof(double);
  cudaError_t e = cudaMalloc(&d, 2 * bytes);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CAVITY_ERR_OOM : CAVITY_ERR_CUDA;
  std::vector<double> rel((size_t)n);
  e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_check_sqrt<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(rel.data(), d + n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return CAVITY_ERR_CUDA;
  double m = 0.0;
  long long nd = 0;
  for (double r : rel) {
    m = std::max(m, r);
    nd += r != 0.0;
  }
  *max_rel = m;
  *n_diff = nd;
  return CAVITY_OK;
}

int cavity_test_wait_timeout(cavity_t *h, long long wait_cycles, int withhold_plane) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  if (!h->f32) return fail(h, CAVITY_ERR_UNSUPPORTED, "bounded waits exist in the FP32-mixed step only");
  if (wait_cycles < 1000 || wait_cycles > kWaitCycles || withhold_plane < -1)
    return fail(h, CAVITY_ERR_INVALID_ARG, "wait limit outside [1000, 4e9] cycles or plane < -1");
  DeviceGuard g(h->dev);
  CK(cudaStreamSynchronize(h->stream));
  h->wait_cycles = wait_cycles;
  h->withhold_plane = withhold_plane;
  return build_graphs(h);
}

int cavity_measure_fp64_peak(int device, double *tflops) {
  if (!tflops) return CAVITY_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(device);
  cavity *h = nullptr;  // no handle: CK reports the code only
  int sms = 0, per_sm = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_peak, kDfmaThreads, 0));
  const int grid = sms * std::max(per_sm, 1);
  const int iters = 4096;
  double *sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CAVITY_OK;
  float best = 0.f;
  if (cudaMalloc(&sink, sizeof(double) * grid) != cudaSuccess) return CAVITY_ERR_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = CAVITY_ERR_CUDA;
  } else {
    const double a = 1.0 - 1.0 / 1048576.0, b = 1.0 / 1048576.0;
    k_dfma_peak<<<grid, kDfmaThreads, 0, st>>>(sink, iters / 8, a, b);  // warm-up
    for (int rep = 0; rep < 3 && rc == CAVITY_OK; ++rep) {
      cudaEventRecord(e0, st);
      k_dfma_peak<<<grid, kDfmaThreads, 0, st>>>(sink, iters, a, b);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = CAVITY_ERR_CUDA;
        break;
      }
      if (best == 0.f || ms < best) best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  if (rc != CAVITY_OK) return rc;
  const double flops = 2.0 * kDfmaChains * kDfmaUnroll * (double)iters * grid * kDfmaThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return CAVITY_OK;
}

int cavity_sync(cavity_t *h) {
  if (!h) return CAVITY_ERR_INVALID_ARG;
  DeviceGuard g(h->dev);
  return all_status(h);
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
