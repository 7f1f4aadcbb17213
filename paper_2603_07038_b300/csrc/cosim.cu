// C-ABI implementation of libcosim (see include/cosim.h): context state,
// device allocation, derived tables and the launch sequence of every call.
#include "../../include/cosim.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "common.cuh"
#include "em.cuh"
#include "mech.cuh"
#include "thermal.cuh"

using namespace cosim;

namespace {

// EM tile: 31 x (TY-1) owned nodes per CTA of 32 x TY threads. TY = 8 always
// exists; FP32 plain steps may also use TY = 4 (more, smaller CTAs for small
// grids), chosen per grid shape by cosim_autotune.
constexpr int kEmTX = 32, kEmTY = 8, kEmTYSmall = 4;
constexpr int em_ty_index(int ty) { return ty == kEmTY ? 0 : 1; }
constexpr int kMvTX = 32, kMvTY = 8;  // matvec tile
constexpr int kRedBlocks = 1184;      // fixed grid of the vector kernels (8 x 148)
// dynamic shared memory a kernel may opt in to: the 227 KB of a CTA less
// 1 KB for its static shared variables
constexpr size_t kMaxSmemOptin = 232448 - 1024;
constexpr uint32_t kEmFlags = COSIM_ACCUM_JOULE | COSIM_COUPLED_THERMAL | COSIM_COUPLED_FUSED;
constexpr int kSrcPadLo = 4, kSrcPadHi = 16;  // zero ints around the source-row offsets
thread_local std::string g_create_error;

}  // namespace

struct cosim_ctx {
  // problem
  int nx = 0, ny = 0, nz = 0, px = 0;
  long long plane = 0, npad = 0;  // padded node-array length
  int prec = COSIM_FP32;
  size_t rsz = 4;
  std::vector<double> h[3];
  std::vector<cosim_material> mats;
  int em_bc[6] = {0, 0, 0, 0, 0, 0};
  int L = 0;
  double cpml_order = 3, cpml_eps_r = 1, h_conv[6] = {0, 0, 0, 0, 0, 0}, T_amb = 300, T_init = 300;
  double dt = 0, dt_th_limit = -1, thermal_safety = 0.9;
  cudaStream_t stream = nullptr;
  // asynchronous field reads: staging buffer, copy stream, events
  void *rd_stage = nullptr;
  size_t rd_bytes = 0;
  cudaStream_t rd_stream = nullptr;
  cudaEvent_t rd_packed = nullptr, rd_done = nullptr;
  bool rd_pending = false;
  cosim_allocator alloc{};
  bool has_alloc = false;
  // device memory
  std::vector<std::pair<void *, size_t>> allocs;
  size_t bytes = 0;
  uint8_t *mat = nullptr;
  void *dh[3]{}, *dih[3]{}, *didual[3]{};
  void *mtab = nullptr, *cpml = nullptr;
  void *E[2][3]{}, *H[2][3]{};
  // CPML state per parity / derivative axis / slot: chi = dF + psi and dF of the previous step;
  // FP32 contexts also hold the low part of chi (lE, lH)
  void *xE[2][3][2]{}, *dE[2][3][2]{}, *xH[2][3][2]{}, *dH[2][3][2]{};
  void *lE[2][3][2]{}, *lH[2][3][2]{};
  // TMA descriptors of E, H (per parity and component) and the Joule window
  // per EM tile height (index em_ty_index): boxes of TY or TY + 1 rows
  CUtensorMap tmE[2][2][3], tmH[2][2][3], tmQ[2], tmT[2][2];
  // the same for the interior tile pairs (boxes em2_box_x wide)
  CUtensorMap tmE2[2][2][3], tmH2[2][2][3], tmQ2[2], tmT2[2][2];
  int *dev_err = nullptr;  // device word: a bounded in-kernel wait gave up
  long long wait_cycles = kWaitCycles;  // the bound of those waits (cosim_set_option)
  int slo[3]{}, shi[3]{}, sn[3]{};
  long long psi_len[3]{};
  int par = 0;
  long long step = 0, n_acc = 0;
  long long *dstep = nullptr;  // device copy of the source time index (advanced per call)
  // captured EM graph (cosim_em_graph_capture): steps per replay, Joule flag,
  // the E/H parity it starts from, kernels per replay
  cudaGraphExec_t gexec = nullptr;
  int64_t g_nsteps = 0, g_launches = 0;
  bool g_accum = false, g_coupled = false;
  int g_par = 0, g_tpar = 0;
  long long launches = 0;  // kernels launched by this context
  long long src_version = 0;  // changes with every cosim_set_sources
  // peak-temperature snapshots of the coupled marching (cosim_coupled_march):
  // pk[5] (see peak_check_kernel), the snapshot of T at the recorded peak,
  // the check interval (0: not tracking) and the step count tracking started at
  unsigned long long *pk = nullptr;
  void *T_peak = nullptr;
  int64_t pk_check_every = 0;
  long long pk_base = 0;
  double *Q = nullptr;      // Joule energy per node, FP64
  void *Qs = nullptr;       // short-window Joule accumulator (context precision)
  bool qs_dirty = false;    // Qs may hold energy not yet folded into Q
  void *T[2]{};
  int tpar = 0;
  void *P = nullptr;
  void *scratch = nullptr;  // npad doubles: staging and per-node temporaries
  double *part = nullptr;   // reduction partials, 3 x kRedBlocks (+ matvec CTAs)
  int npart = 0;
  double *scal = nullptr;   // misc device scalars
  double *host_scal = nullptr;  // pinned
  // sources
  int *src_row = nullptr;       // = src_row_buf + kSrcPadLo
  int *src_row_buf = nullptr;   // allocation: kSrcPadLo zeros, the offsets, kSrcPadHi zeros
  CUtensorMap tmV[2], tmV2[2];  // voxel IDs (x, y, z), boxes em_vox_box_x / em2_vox_box_x x (TY+1) x 1 per tile height
  int em_ty = kEmTY;   // EM tile height of FP32 plain steps
  int th_by = 0;       // thermal step kernel: 0 = TMA-staged tiles, 4/8/16 = classic block height
  CUtensorMap thT[2][2], thP[2], thV[2];  // the TMA thermal kernel's T (per tile width, buffer), P and voxel boxes
  int th_np = 1;                           // node pairs per thread of the TMA thermal kernel (1 or 2)
  // the TMA matvec's boxes: the two CG direction buffers (Pv, Pv2), the
  // residual, the inverse diagonal, the constraint bits, the voxels
  CUtensorMap mvU[2][3], mvR[3], mvD[3], mvM, mvV;
  void *zt = nullptr;  // per node plane k: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1) (zero outside)
  int vpx = 0;         // voxel row pitch
  int4 *src_ent = nullptr;
  void *src_amp = nullptr;
  long long amp_len = 0;
  // mechanics (allocated on first use)
  bool mech_ready = false;
  uint8_t *mask = nullptr;
  void *U[3]{}, *F[3]{}, *Rv[3]{}, *Pv[3]{}, *Pv2[3]{}, *Qv[3]{}, *Dinv[3]{};  // Pv2: the other direction buffer
  void *VM = nullptr, *UMAG = nullptr;
  CgScalars *cg = nullptr;
  // FP64 geometry (aliases of the tables above for FP64 contexts) and the
  // FP64 vectors of the mixed-precision refinement (allocated on first use)
  void *dh64[3]{}, *dih64[3]{}, *didual64[3]{}, *mtab64 = nullptr;
  bool refine_ready = false;
  double *U64[3]{}, *F64[3]{}, *R64[3]{};
  std::string err;
};

// ---------------------------------------------------------------- helpers

#define CHECK_CUDA(ctx, call)                                                          \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return COSIM_ERR_CUDA;                                                           \
    }                                                                                  \
  } while (0)

#define CHECK_LAUNCH(ctx) CHECK_CUDA(ctx, cudaGetLastError())

static cosim_status fail(cosim_ctx *c, cosim_status s, const std::string &msg) {
  c->err = msg;
  return s;
}

static cosim_status dev_alloc(cosim_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return COSIM_OK;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->has_alloc) {
    *p = c->alloc.alloc(bytes, c->alloc.user);
    if (*p == nullptr) return fail(c, COSIM_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(c, COSIM_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  c->allocs.emplace_back(*p, bytes);
  c->bytes += bytes;
  cudaError_t e = cudaMemsetAsync(*p, 0, bytes, c->stream);
  if (e != cudaSuccess) return fail(c, COSIM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  return COSIM_OK;
}

#define ALLOC(ctx, ptr, bytes)                                        \
  do {                                                                \
    cosim_status s_ = dev_alloc((ctx), (void **)&(ptr), (bytes));     \
    if (s_ != COSIM_OK) return s_;                                    \
  } while (0)

template <typename R>
static Geo<R> make_geo(const cosim_ctx *c) {
  Geo<R> g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  g.px = c->px;
  g.plane = c->plane;
  g.mat = c->mat;
  g.vpx = c->vpx;
  for (int a = 0; a < 3; ++a) {
    g.h[a] = (const R *)c->dh[a];
    g.ih[a] = (const R *)c->dih[a];
    g.idual[a] = (const R *)c->didual[a];
  }
  g.mtab = (const R *)c->mtab;
  g.nmat = (int)c->mats.size();
  return g;
}

static int n_of(const cosim_ctx *c, int a) { return a == 0 ? c->nx : (a == 1 ? c->ny : c->nz); }

// host -> device copy ordered on the context stream (pageable sources are
// staged by the driver before the call returns)
static cosim_status h2d(cosim_ctx *c, void *dst, const void *src, size_t bytes) {
  CHECK_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  return COSIM_OK;
}

// upload a host double array converted to the context precision
static cosim_status upload_real(cosim_ctx *c, void **dst, const std::vector<double> &v) {
  ALLOC(c, *dst, v.size() * c->rsz);
  if (c->prec == COSIM_FP64) return h2d(c, *dst, v.data(), v.size() * 8);
  std::vector<float> f(v.begin(), v.end());
  cosim_status st = h2d(c, *dst, f.data(), f.size() * 4);
  if (st == COSIM_OK) CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

// upload a host double array as FP64
static cosim_status upload_f64(cosim_ctx *c, void **dst, const std::vector<double> &v) {
  ALLOC(c, *dst, v.size() * 8);
  cosim_status st = h2d(c, *dst, v.data(), v.size() * 8);
  if (st == COSIM_OK) CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

static Geo<double> make_geo64(const cosim_ctx *c) {
  Geo<double> g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  g.px = c->px;
  g.plane = c->plane;
  g.mat = c->mat;
  g.vpx = c->vpx;
  for (int a = 0; a < 3; ++a) {
    g.h[a] = (const double *)c->dh64[a];
    g.ih[a] = (const double *)c->dih64[a];
    g.idual[a] = (const double *)c->didual64[a];
  }
  g.mtab = (const double *)c->mtab64;
  g.nmat = (int)c->mats.size();
  return g;
}

// CPML conductivity profile (kappa = 1, alpha = 0), polynomial grading of
// order m inside each layer, sigma_max = 0.8 (m+1) / (eta0 * mean cell * sqrt(eps_r_bg)).
static double cpml_sigma(const cosim_ctx *c, int a, double pos, const std::vector<double> &x) {
  const int n = n_of(c, a), L = c->L;
  const double m = c->cpml_order, eta0 = std::sqrt(kMu0 / kEps0);
  double sig = 0;
  if (L > 0 && c->em_bc[2 * a] == COSIM_BC_CPML) {
    const double xi = x[L], d = x[L] - x[0];
    if (pos < xi) sig = 0.8 * (m + 1) / (eta0 * (d / L) * std::sqrt(c->cpml_eps_r)) * std::pow((xi - pos) / d, m);
  }
  if (L > 0 && c->em_bc[2 * a + 1] == COSIM_BC_CPML) {
    const double xi = x[n - L], d = x[n] - x[n - L];
    if (pos > xi) sig = 0.8 * (m + 1) / (eta0 * (d / L) * std::sqrt(c->cpml_eps_r)) * std::pow((pos - xi) / d, m);
  }
  return sig;
}

// ---------------------------------------------------------------- create

constexpr size_t kHostVoxelCheck = (size_t)1 << 24;  // voxels checked on the host (larger grids: on the device)

// the largest voxel ID of the pitched voxel array (rows of nx IDs, pitch vpx)
__global__ void __launch_bounds__(256) voxel_max_kernel(const uint8_t *mat, int nx, long long rows, int vpx,
                                                        unsigned *out) {
  unsigned mx = 0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) mx = max(mx, (unsigned)mat[r * vpx + i]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx != 0) atomicMax(out, mx);
}

static cosim_status validate(const cosim_grid_desc *d, const cosim_options *o, std::string &why) {
  if (!d) return why = "desc is NULL", COSIM_ERR_INVALID;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return why = "grid sizes must be >= 1", COSIM_ERR_INVALID;
  if ((long long)(d->nx + 1) * (d->ny + 1) * (d->nz + 1) > (1LL << 36))
    return why = "grid too large", COSIM_ERR_INVALID;
  if (!d->dx || !d->dy || !d->dz || !d->mat || !d->mats) return why = "NULL array in desc", COSIM_ERR_INVALID;
  if (d->nmat < 1 || d->nmat > kMaxMat) return why = "nmat must be in [1, 256]", COSIM_ERR_INVALID;
  const double *hs[3] = {d->dx, d->dy, d->dz};
  const int ns[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; ++a)
    for (int p = 0; p < ns[a]; ++p)
      if (!(hs[a][p] > 0) || !std::isfinite(hs[a][p])) return why = "cell sizes must be finite and > 0", COSIM_ERR_INVALID;
  for (int m = 0; m < d->nmat; ++m) {
    const cosim_material &q = d->mats[m];
    if (!(q.eps_r > 0) || !(q.mu_r > 0) || q.sigma0 < 0 || !(q.k >= 0) || !(q.rho_cp > 0) || !(q.E > 0) ||
        !(q.nu > -1 && q.nu < 0.5))
      return why = "material " + std::to_string(m) + " has out-of-range constants", COSIM_ERR_INVALID;
  }
  // Every voxel ID below nmat. Grids up to kHostVoxelCheck voxels are checked
  // here, before any device work; larger ones on the device after the
  // upload (a host pass over a full package's 134 M IDs took milliseconds of
  // every cosim_create).
  if (d->nmat < 256 && (size_t)d->nx * d->ny * d->nz <= kHostVoxelCheck) {
    const size_t nc = (size_t)d->nx * d->ny * d->nz;
    uint8_t mx = 0;
    for (size_t q = 0; q < nc; ++q) mx = d->mat[q] > mx ? d->mat[q] : mx;
    if (mx >= d->nmat) return why = "voxel material id >= nmat", COSIM_ERR_INVALID;
  }
  bool any_cpml = false;
  for (int f = 0; f < 6; ++f) {
    if (d->em_bc[f] < 0 || d->em_bc[f] > 2) return why = "bad em_bc", COSIM_ERR_INVALID;
    if (d->em_bc[f] == COSIM_BC_CPML) any_cpml = true;
    if (d->h_conv[f] < 0) return why = "h_conv must be >= 0", COSIM_ERR_INVALID;
  }
  if (any_cpml) {
    if (d->cpml_cells < 1 || d->cpml_cells > kMaxL) return why = "cpml_cells must be in [1, 32]", COSIM_ERR_INVALID;
    if (!(d->cpml_eps_r > 0) || !(d->cpml_order >= 0)) return why = "bad CPML grading", COSIM_ERR_INVALID;
    for (int a = 0; a < 3; ++a) {
      const int layers = (d->em_bc[2 * a] == COSIM_BC_CPML) + (d->em_bc[2 * a + 1] == COSIM_BC_CPML);
      if (layers > 0 && ns[a] < layers * d->cpml_cells + 2)
        return why = "an axis needs >= (CPML faces x cpml_cells) + 2 cells", COSIM_ERR_INVALID;
    }
  }
  if (o && o->precision != COSIM_FP64 && o->precision != COSIM_FP32) return why = "bad precision", COSIM_ERR_INVALID;
  return COSIM_OK;
}

template <typename R>
static cudaError_t set_smem_limits() {
  const int mv = (kMaxMat * M_COLS + 2 * 3 * (kMvTY + 1) * (kMvTX + 1) + 24 * kMvTY * kMvTX) * (int)sizeof(R);
  cudaError_t e =
      cudaFuncSetAttribute(hex8_matvec_kernel<R, kMvTX, kMvTY>, cudaFuncAttributeMaxDynamicSharedMemorySize, mv);
  if (e != cudaSuccess) return e;
  const int em = (int)em_smem_bytes<R, kEmTY>(kMaxMat);
  const void *kernels[6] = {(const void *)em_step_kernel<R, int, kEmTX, kEmTY, false, false>,
                            (const void *)em_step_kernel<R, long long, kEmTX, kEmTY, false, false>,
                            (const void *)em_step_kernel<R, int, kEmTX, kEmTY, true, false>,
                            (const void *)em_step_kernel<R, long long, kEmTX, kEmTY, true, false>,
                            (const void *)em_step_kernel<R, int, kEmTX, kEmTY, true, true>,
                            (const void *)em_step_kernel<R, long long, kEmTX, kEmTY, true, true>};
  for (const void *k : kernels)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, em)) != cudaSuccess) return e;
  const void *batch[2] = {(const void *)em_batch_kernel<R, int, kEmTX, kEmTY>,
                          (const void *)em_batch_kernel<R, long long, kEmTX, kEmTY>};
  for (const void *k : batch)
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, em)) != cudaSuccess) return e;
  const int mvt = (int)std::min(mv_smem_bytes<R, kMvTY, false>(kMaxMat), kMaxSmemOptin);
  const int mvd = (int)std::min(mv_smem_bytes<R, kMvTY, true>(kMaxMat), kMaxSmemOptin);
  if ((e = cudaFuncSetAttribute(hex8_matvec_tma_kernel<R, kMvTY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                mvt)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(hex8_matvec_tma_kernel<R, kMvTY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                mvd)) != cudaSuccess)
    return e;
  const int th1 = (int)(th_stage_offset<R>(kMaxMat) + kThStages * sizeof(ThStage<R, 1>) + 128);
  const int th2 = (int)(th_stage_offset<R>(kMaxMat) + kThStages * sizeof(ThStage<R, 2>) + 128);
  if ((e = cudaFuncSetAttribute(thermal_tma_kernel<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, th1)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(thermal_tma_kernel<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, th2)) !=
          cudaSuccess)
    return e;
  if constexpr (sizeof(R) == 4) {
    const int em4 = (int)em_smem_bytes<R, kEmTYSmall>(kMaxMat);
    const void *small[2] = {(const void *)em_step_kernel<R, int, kEmTX, kEmTYSmall, false, false>,
                            (const void *)em_step_kernel<R, long long, kEmTX, kEmTYSmall, false, false>};
    for (const void *k : small)
      if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, em4)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// TMA descriptor of a padded node array (x fastest, pitch px, planes of
// px (ny+1)): extents nx+1, ny+1, nz+1 (reads past them return zero), box of
// em_box_x x rows x 1 nodes for the EM kernel's plane staging.
static cosim_status encode_map(cosim_ctx *c, CUtensorMap *m, CUtensorMapDataType type, int rank, void *base,
                               const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return fail(c, COSIM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  }
  const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = encode(m, type, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, COSIM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return COSIM_OK;
}
static cosim_status encode_node_map(cosim_ctx *c, CUtensorMap *m, void *base, int rows, int cols = em_box_x<kEmTX>()) {
  const cuuint64_t dims[3] = {(cuuint64_t)c->nx + 1, (cuuint64_t)c->ny + 1, (cuuint64_t)c->nz + 1};
  const cuuint64_t strides[2] = {(cuuint64_t)c->px * c->rsz, (cuuint64_t)c->plane * c->rsz};
  const cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)rows, 1};
  return encode_map(c, m, c->rsz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
                    dims, strides, box);
}
// voxel IDs: (x, y, z) = (nx, ny, nz) bytes with row pitch vpx
static cosim_status encode_voxel_map(cosim_ctx *c, CUtensorMap *m, int rows, int cols = em_vox_box_x<kEmTX>()) {
  const cuuint64_t dims[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz};
  const cuuint64_t strides[2] = {(cuuint64_t)c->vpx, (cuuint64_t)c->vpx * c->ny};
  const cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)rows, 1};
  return encode_map(c, m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, c->mat, dims, strides, box);
}


static void free_one(cosim_ctx *c, void *p);

static cosim_status create_impl(cosim_ctx *c, const cosim_grid_desc *d, const cosim_options *o) {
  c->nx = d->nx;
  c->ny = d->ny;
  c->nz = d->nz;
  c->px = ((d->nx + 1) + 31) / 32 * 32;
  c->plane = (long long)c->px * (d->ny + 1);
  c->npad = c->plane * (d->nz + 1);
  c->prec = o ? o->precision : COSIM_FP32;
  c->rsz = c->prec == COSIM_FP64 ? 8 : 4;
  c->stream = o ? (cudaStream_t)o->stream : nullptr;
  if (o && o->allocator && o->allocator->alloc && o->allocator->free) {
    c->alloc = *o->allocator;
    c->has_alloc = true;
  }
  c->thermal_safety = (o && o->thermal_safety > 0) ? o->thermal_safety : 0.9;
  c->h[0].assign(d->dx, d->dx + d->nx);
  c->h[1].assign(d->dy, d->dy + d->ny);
  c->h[2].assign(d->dz, d->dz + d->nz);
  c->mats.assign(d->mats, d->mats + d->nmat);
  for (int f = 0; f < 6; ++f) {
    c->em_bc[f] = d->em_bc[f];
    c->h_conv[f] = d->h_conv[f];
  }
  bool any_cpml = false;
  for (int f = 0; f < 6; ++f) any_cpml |= d->em_bc[f] == COSIM_BC_CPML;
  c->L = any_cpml ? d->cpml_cells : 0;
  c->cpml_order = d->cpml_order;
  c->cpml_eps_r = d->cpml_eps_r;
  c->T_amb = d->T_amb;
  c->T_init = d->T_init;

  // EM step: Courant limit of the finest cells at the fastest wave speed
  double vmax = 0;
  for (auto &m : c->mats) vmax = std::max(vmax, 1.0 / std::sqrt(kEps0 * m.eps_r * kMu0 * m.mu_r));
  double s = 0;
  for (int a = 0; a < 3; ++a) {
    const double hmin = *std::min_element(c->h[a].begin(), c->h[a].end());
    s += 1.0 / (hmin * hmin);
  }
  const double cfl = (o && o->cfl > 0) ? o->cfl : 0.99;
  c->dt = (o && o->dt_em > 0) ? o->dt_em : cfl / (vmax * std::sqrt(s));

  // geometry tables
  for (int a = 0; a < 3; ++a) {
    const int n = n_of(c, a);
    std::vector<double> ih(n), idual(n + 1);
    for (int p = 0; p < n; ++p) ih[p] = 1.0 / c->h[a][p];
    for (int p = 0; p <= n; ++p) {
      const double dl = (p > 0 ? 0.5 * c->h[a][p - 1] : 0.0) + (p < n ? 0.5 * c->h[a][p] : 0.0);
      idual[p] = 1.0 / dl;
    }
    cosim_status st;
    if ((st = upload_real(c, &c->dh[a], c->h[a])) != COSIM_OK) return st;
    if ((st = upload_real(c, &c->dih[a], ih)) != COSIM_OK) return st;
    if ((st = upload_real(c, &c->didual[a], idual)) != COSIM_OK) return st;
    // FP64 copies for the mixed-precision stress refinement
    if (c->prec == COSIM_FP64) {
      c->dh64[a] = c->dh[a];
      c->dih64[a] = c->dih[a];
      c->didual64[a] = c->didual[a];
    } else {
      if ((st = upload_f64(c, &c->dh64[a], c->h[a])) != COSIM_OK) return st;
      if ((st = upload_f64(c, &c->dih64[a], ih)) != COSIM_OK) return st;
      if ((st = upload_f64(c, &c->didual64[a], idual)) != COSIM_OK) return st;
    }
  }
  // material table, plus an all-zero row (index nmat) that the EM kernel uses
  // for voxels outside the grid
  std::vector<double> mt((c->mats.size() + 1) * M_COLS, 0.0);
  for (size_t m = 0; m < c->mats.size(); ++m) {
    const cosim_material &q = c->mats[m];
    const double lam = q.E * q.nu / ((1 + q.nu) * (1 - 2 * q.nu)), mu = q.E / (2 * (1 + q.nu));
    double *r = &mt[m * M_COLS];
    r[M_EPS] = kEps0 * q.eps_r;
    r[M_SDT2] = q.sigma0 * c->dt * 0.5;
    r[M_IMU] = 1.0 / (kMu0 * q.mu_r);
    r[M_K] = q.k;
    r[M_RHOCP] = q.rho_cp;
    r[M_LAM] = lam;
    r[M_MU] = mu;
    r[M_BETA] = (3 * lam + 2 * mu) * q.alpha_L;
    r[M_TCR] = q.tcr;
    r[M_TC0] = 1.0 + q.tcr * (c->T_init - q.T0);
  }
  mt[c->mats.size() * M_COLS + M_TC0] = 1.0;  // the zero row: sigma(T) = 0 / 1
  cosim_status st;
  if ((st = upload_real(c, &c->mtab, mt)) != COSIM_OK) return st;
  if (c->prec == COSIM_FP64)
    c->mtab64 = c->mtab;
  else if ((st = upload_f64(c, &c->mtab64, mt)) != COSIM_OK)
    return st;
  // voxels: rows padded to a 16-byte pitch (a TMA stride rule); the padding
  // bytes are zero and never read as material
  c->vpx = (c->nx + 15) / 16 * 16;
  ALLOC(c, c->mat, (size_t)c->vpx * c->ny * c->nz);
  CHECK_CUDA(c, cudaMemcpy2DAsync(c->mat, c->vpx, d->mat, c->nx, c->nx, (size_t)c->ny * c->nz,
                                  cudaMemcpyHostToDevice, c->stream));
  if (d->nmat < 256 && (size_t)d->nx * d->ny * d->nz > kHostVoxelCheck) {  // the largest voxel ID, on the device
    unsigned *dmax = nullptr;
    ALLOC(c, dmax, sizeof(unsigned));
    voxel_max_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->mat, c->nx, (long long)c->ny * c->nz, c->vpx, dmax);
    ++c->launches;
    CHECK_LAUNCH(c);
    unsigned mx = 0;
    CHECK_CUDA(c, cudaMemcpyAsync(&mx, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    free_one(c, dmax);
    if (mx >= (unsigned)d->nmat) return fail(c, COSIM_ERR_INVALID, "voxel material id >= nmat");
  }
  // per node plane k: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1), zero where the
  // cell does not exist; one 16/32-byte record copied per plane by the EM kernel
  {
    std::vector<double> zt(4 * (size_t)(c->nz + 1), 0.0);
    for (int k = 0; k <= c->nz; ++k) {
      zt[4 * k + 0] = k < c->nz ? c->h[2][k] : 0.0;
      zt[4 * k + 1] = k < c->nz ? 1.0 / c->h[2][k] : 0.0;
      zt[4 * k + 2] = 1.0 / ((k > 0 ? 0.5 * c->h[2][k - 1] : 0.0) + (k < c->nz ? 0.5 * c->h[2][k] : 0.0));
      zt[4 * k + 3] = k > 0 ? c->h[2][k - 1] : 0.0;
    }
    if ((st = upload_real(c, &c->zt, zt)) != COSIM_OK) return st;
  }

  // CPML slabs and the table of 1 - b per [axis][E,H][kMaxSlab]
  std::vector<double> cp(kCpmlTable);
  for (int a = 0; a < 3; ++a) {
    const int n = n_of(c, a);
    c->slo[a] = (c->L > 0 && c->em_bc[2 * a] == COSIM_BC_CPML) ? c->L : 0;
    c->shi[a] = (c->L > 0 && c->em_bc[2 * a + 1] == COSIM_BC_CPML) ? c->L : 0;
    const int base = c->slo[a] > 0 ? c->slo[a] + 1 : 0;
    c->sn[a] = base + (c->shi[a] > 0 ? c->shi[a] + 1 : 0);
    std::vector<double> x(n + 1, 0.0);
    for (int p = 0; p < n; ++p) x[p + 1] = x[p] + c->h[a][p];
    for (int sidx = 0; sidx < kMaxSlab; ++sidx)
      for (int type = 0; type < 2; ++type) {
        double omb = 0;  // 1 - b, b = exp(-sigma dt / eps0); c = b - 1 (kappa = 1, alpha = 0)
        if (sidx < c->sn[a]) {
          const int p = sidx < base ? sidx : (n - c->shi[a]) + (sidx - base);
          const bool ok = type == 0 ? (p <= n) : (p < n);
          if (ok) {
            const double pos = type == 0 ? x[p] : 0.5 * (x[p] + x[p + 1]);
            const double sig = cpml_sigma(c, a, pos, x);
            if (sig > 0) omb = -std::expm1(-sig * c->dt / kEps0);
          }
        }
        cp[(a * 2 + type) * kMaxSlab + sidx] = omb;
      }
  }
  if ((st = upload_real(c, &c->cpml, cp)) != COSIM_OK) return st;
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  c->psi_len[0] = (long long)(c->nz + 1) * (c->ny + 1) * c->sn[0];
  c->psi_len[1] = (long long)(c->nz + 1) * c->sn[1] * c->px;
  c->psi_len[2] = (long long)c->sn[2] * (c->ny + 1) * c->px;

  // fields
  for (int p = 0; p < 2; ++p)
    for (int a = 0; a < 3; ++a) {
      ALLOC(c, c->E[p][a], c->npad * c->rsz);
      ALLOC(c, c->H[p][a], c->npad * c->rsz);
      for (int s2 = 0; s2 < 2; ++s2)
        if (c->psi_len[a] > 0 && a < 2) {  // x / y slabs: one 16-byte record per element
          ALLOC(c, c->xE[p][a][s2], c->psi_len[a] * 16);
          ALLOC(c, c->xH[p][a][s2], c->psi_len[a] * 16);
        } else if (c->psi_len[a] > 0) {  // z slab: chi (high part), previous derivative, chi low part
          ALLOC(c, c->xE[p][a][s2], c->psi_len[a] * c->rsz);
          ALLOC(c, c->dE[p][a][s2], c->psi_len[a] * c->rsz);
          ALLOC(c, c->xH[p][a][s2], c->psi_len[a] * c->rsz);
          ALLOC(c, c->dH[p][a][s2], c->psi_len[a] * c->rsz);
          if (c->rsz == 4) {
            ALLOC(c, c->lE[p][a][s2], c->psi_len[a] * c->rsz);
            ALLOC(c, c->lH[p][a][s2], c->psi_len[a] * c->rsz);
          }
        }
    }
  ALLOC(c, c->Q, c->npad * 8);
  ALLOC(c, c->Qs, c->npad * c->rsz);
  ALLOC(c, c->dev_err, sizeof(int));
  ALLOC(c, c->dstep, sizeof(long long));
  for (int t = 0; t < 2; ++t) {
    const int ty = t == 0 ? kEmTY : kEmTYSmall;
    for (int p = 0; p < 2; ++p)
      for (int a = 0; a < 3; ++a) {
        if ((st = encode_node_map(c, &c->tmE[t][p][a], c->E[p][a], ty + 1)) != COSIM_OK) return st;
        if ((st = encode_node_map(c, &c->tmH[t][p][a], c->H[p][a], ty)) != COSIM_OK) return st;
        if ((st = encode_node_map(c, &c->tmE2[t][p][a], c->E[p][a], ty + 1, em2_box_x())) != COSIM_OK) return st;
        if ((st = encode_node_map(c, &c->tmH2[t][p][a], c->H[p][a], ty, em2_box_x())) != COSIM_OK) return st;
      }
    if ((st = encode_node_map(c, &c->tmQ[t], c->Qs, ty)) != COSIM_OK) return st;
    if ((st = encode_voxel_map(c, &c->tmV[t], ty + 1)) != COSIM_OK) return st;
    if ((st = encode_node_map(c, &c->tmQ2[t], c->Qs, ty, em2_box_x())) != COSIM_OK) return st;
    if ((st = encode_voxel_map(c, &c->tmV2[t], ty + 1, em2_vox_box_x())) != COSIM_OK) return st;
  }
  ALLOC(c, c->T[0], c->npad * c->rsz);
  ALLOC(c, c->T[1], c->npad * c->rsz);
  ALLOC(c, c->P, c->npad * c->rsz);
  for (int t = 0; t < 2; ++t)
    for (int p = 0; p < 2; ++p)
      if ((st = encode_node_map(c, &c->tmT[t][p], c->T[p], (t == 0 ? kEmTY : kEmTYSmall) + 1)) != COSIM_OK ||
          (st = encode_node_map(c, &c->tmT2[t][p], c->T[p], (t == 0 ? kEmTY : kEmTYSmall) + 1, em2_box_x())) !=
              COSIM_OK)
        return st;
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q)
      if ((st = encode_node_map(c, &c->thT[q][p], c->T[p], kThTY + 2, th_box_t(q + 1))) != COSIM_OK) return st;
  for (int q = 0; q < 2; ++q) {
    if ((st = encode_node_map(c, &c->thP[q], c->P, kThTY, th_tx(q + 1))) != COSIM_OK) return st;
    if ((st = encode_voxel_map(c, &c->thV[q], kThTY + 1, th_box_v(q + 1))) != COSIM_OK) return st;
  }
  // two node pairs per thread once their grid fills the GPU about two and a
  // half times at two CTAs per SM (measured crossover near 768 x 768 nodes);
  // one pair (three CTAs per SM) on smaller grids
  {
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long ctas2 = (long long)((c->nx + 1 + th_tx(2) - 1) / th_tx(2)) * ((c->ny + 1 + kThTY - 1) / kThTY);
    c->th_np = ctas2 >= 5LL * nsm ? 2 : 1;
  }
  ALLOC(c, c->scratch, c->npad * 8);
  const int mv_blocks = ((c->nx + 1) + kMvTX - 2) / (kMvTX - 1) * (((c->ny + 1) + kMvTY - 2) / (kMvTY - 1));
  c->npart = std::max(kRedBlocks, mv_blocks);
  ALLOC(c, c->part, 3 * (size_t)c->npart * 8);
  ALLOC(c, c->scal, 64 * 8);
  CHECK_CUDA(c, cudaMallocHost((void **)&c->host_scal, 64 * 8));
  // the device holds the temperature rise T - T_init (zero after the memset):
  // full relative precision for small Joule heating even in FP32
  CHECK_CUDA(c, set_smem_limits<double>());
  CHECK_CUDA(c, set_smem_limits<float>());
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return COSIM_OK;
}

extern "C" cosim_status cosim_create(const cosim_grid_desc *desc, const cosim_options *opts, cosim_ctx **out) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return COSIM_ERR_INVALID;
  }
  *out = nullptr;
  std::string why;
  cosim_status st = validate(desc, opts, why);
  if (st != COSIM_OK) {
    g_create_error = why;
    return st;
  }
  cosim_ctx *c = new cosim_ctx();
  st = create_impl(c, desc, opts);
  if (st != COSIM_OK) {
    g_create_error = c->err;
    cosim_destroy(c);
    return st;
  }
  *out = c;
  return COSIM_OK;
}

static void drop_graph(cosim_ctx *c);

extern "C" void cosim_destroy(cosim_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->rd_stream) {
    cudaStreamSynchronize(c->rd_stream);
    cudaEventDestroy(c->rd_packed);
    cudaEventDestroy(c->rd_done);
    cudaStreamDestroy(c->rd_stream);
  }
  drop_graph(c);
  for (auto &a : c->allocs) {
    if (c->has_alloc)
      c->alloc.free(a.first, c->alloc.user);
    else
      cudaFree(a.first);
  }
  if (c->host_scal) cudaFreeHost(c->host_scal);
  delete c;
}

extern "C" const char *cosim_last_error(const cosim_ctx *c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

// ---------------------------------------------------------------- sources

static void free_one(cosim_ctx *c, void *p) {
  if (!p) return;
  for (size_t q = 0; q < c->allocs.size(); ++q)
    if (c->allocs[q].first == p) {
      c->bytes -= c->allocs[q].second;
      if (c->has_alloc)
        c->alloc.free(p, c->alloc.user);
      else
        cudaFree(p);
      c->allocs.erase(c->allocs.begin() + q);
      return;
    }
}

extern "C" cosim_status cosim_set_sources(cosim_ctx *c, int32_t n, const cosim_source *src) {
  if (!c) return COSIM_ERR_INVALID;
  if (n < 0 || (n > 0 && !src)) return fail(c, COSIM_ERR_INVALID, "bad source list");
  drop_graph(c);  // a captured graph holds the source table pointers
  ++c->src_version;  // (and so does a design batch)
  struct Ent { int row, i, axis, s; };
  std::vector<Ent> ents;
  long long amp_len = 0;
  for (int s = 0; s < n; ++s) {
    const cosim_source &q = src[s];
    if (q.axis < 0 || q.axis > 2 || q.n_edges < 0 || (q.n_edges > 0 && !q.edge_ijk) || q.nsteps < 0 ||
        (q.nsteps > 0 && !q.amp))
      return fail(c, COSIM_ERR_INVALID, "bad source " + std::to_string(s));
    for (int e = 0; e < q.n_edges; ++e) {
      const int i = q.edge_ijk[3 * e], j = q.edge_ijk[3 * e + 1], k = q.edge_ijk[3 * e + 2];
      const int nn[3] = {i, j, k};
      bool ok = i >= 0 && j >= 0 && k >= 0 && i <= c->nx && j <= c->ny && k <= c->nz && nn[q.axis] < n_of(c, q.axis);
      if (!ok) return fail(c, COSIM_ERR_INVALID, "source edge outside the grid");
      ents.push_back({k * (c->ny + 1) + j, i, q.axis, s});
    }
    amp_len = std::max(amp_len, (long long)q.nsteps);
  }
  cudaStreamSynchronize(c->stream);
  free_one(c, c->src_row_buf);
  free_one(c, c->src_ent);
  free_one(c, c->src_amp);
  c->src_row = nullptr;
  c->src_row_buf = nullptr;
  c->src_ent = nullptr;
  c->src_amp = nullptr;
  c->amp_len = 0;
  if (ents.empty()) return COSIM_OK;
  const int nrow = (c->nz + 1) * (c->ny + 1);
  std::vector<int> row(nrow + 1, 0);
  for (auto &e : ents) row[e.row + 1]++;
  for (int r = 0; r < nrow; ++r) row[r + 1] += row[r];
  std::vector<int4> ent(ents.size());
  std::vector<int> fill(row.begin(), row.end() - 1);
  for (auto &e : ents) ent[fill[e.row]++] = make_int4(e.i, e.axis, e.s, 0);
  std::vector<double> amp((size_t)n * amp_len, 0.0);
  for (int s = 0; s < n; ++s)
    for (long long t = 0; t < src[s].nsteps; ++t) amp[(size_t)s * amp_len + t] = src[s].amp[t];
  // padded so that the EM kernel's 16-byte aligned bulk copy of the rows
  // j0 .. j0+TY of a plane (start rounded down to 4 entries, from j0 = -1)
  // stays inside the allocation
  ALLOC(c, c->src_row_buf, (row.size() + kSrcPadLo + kSrcPadHi) * sizeof(int));
  c->src_row = c->src_row_buf + kSrcPadLo;
  ALLOC(c, c->src_ent, ent.size() * sizeof(int4));
  cosim_status st;
  if ((st = h2d(c, c->src_row, row.data(), row.size() * sizeof(int))) != COSIM_OK) return st;
  if ((st = h2d(c, c->src_ent, ent.data(), ent.size() * sizeof(int4))) != COSIM_OK) return st;
  if ((st = upload_real(c, &c->src_amp, amp)) != COSIM_OK) return st;
  c->amp_len = amp_len;
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return COSIM_OK;
}

// ---------------------------------------------------------------- EM


template <typename R>
static ThArgs<R> th_args(cosim_ctx *c);

// One thermal step T[tpar] -> T[tpar ^ 1] with time step dt (tpar is not
// flipped here): th_by = 0 launches the TMA-staged kernel, 4/8/16 the classic
// kernel with that block height. Every choice gives identical results.
template <typename R>
static cosim_status launch_thermal(cosim_ctx *c, R dt, bool count = true, unsigned long long *peak = nullptr) {
  ThArgs<R> A = th_args<R>(c);
  A.dt = dt;
  if (c->th_by == 0 || peak != nullptr) {  // (peak tracking: the TMA kernel, same bits as the others)
    ThTmaArgs<R> T;
    T.a = A;
    T.peak = peak;
    const int q = c->th_np - 1;
    T.tmT = c->thT[q][c->tpar];
    T.tmP = c->thP[q];
    T.tmV = c->thV[q];
    T.err = c->dev_err;
    T.wait = c->wait_cycles;
    const dim3 blk(32, kThTY), grd((c->nx + 1 + th_tx(c->th_np) - 1) / th_tx(c->th_np), (c->ny + 1 + kThTY - 1) / kThTY);
    if (c->th_np == 2) {
      const size_t smem = th_stage_offset<R>((int)c->mats.size()) + kThStages * sizeof(ThStage<R, 2>) + 128;
      thermal_tma_kernel<R, 2><<<grd, blk, smem, c->stream>>>(T);
    } else {
      const size_t smem = th_stage_offset<R>((int)c->mats.size()) + kThStages * sizeof(ThStage<R, 1>) + 128;
      thermal_tma_kernel<R, 1><<<grd, blk, smem, c->stream>>>(T);
    }
  } else {
    const dim3 blk(32, c->th_by), grd((c->nx + 1 + 31) / 32, (c->ny + 1 + c->th_by - 1) / c->th_by);
    thermal_kernel<R, 0><<<grd, blk, (c->mats.size() + 1) * sizeof(typename Pair2<R>::T), c->stream>>>(A);
  }
  CHECK_LAUNCH(c);
  if (count) ++c->launches;
  return COSIM_OK;
}

template <typename R, typename I, int TY, bool CPL, bool TH = false>
static void launch_em(const dim3 &grd, const dim3 &blk, size_t smem, cudaStream_t st, const EmArgs<R> &A) {
  em_step_kernel<R, I, kEmTX, TY, CPL, TH><<<grd, blk, smem, st>>>(A);
}

// coupled: the synchronized marching of Sec. II-A (sigma(T^n) in the EM step,
// then one thermal step with the EM dt and that step's Joule power); fused:
// that thermal step inside the EM launch instead of a launch of its own.
// probe: the autotuner's timing launches: every launch reads the current
// E/H/CPML buffers and writes the spare ones, nothing else changes (no
// parity flip, no accumulation, no counters), so the state stays as it was.
// The step arguments of a context that do not change from step to step:
// geometry, walls, CPML, tiling, sources, Joule accumulator, descriptors of
// the voxels and the Joule window (tile height TY).
template <typename R, int TY>
static EmArgs<R> em_args_base(cosim_ctx *c, bool accum) {
  constexpr int t = em_ty_index(TY);
  EmArgs<R> A{};
  A.g = make_geo<R>(c);
  for (int a = 0; a < 3; ++a) {
    A.slo[a] = c->slo[a];
    A.shi[a] = c->shi[a];
    A.sn[a] = c->sn[a];
    A.fixlo[a] = c->em_bc[2 * a] != COSIM_BC_PMC;
    A.fixhi[a] = c->em_bc[2 * a + 1] != COSIM_BC_PMC;
  }
  A.cpml = (const R *)c->cpml;
  // Tiling (see EmArgs). Interior rows: every thread's node j = j0..j0+TY-1
  // (j0 = b (TY-1) - 1) satisfies slo < j < ny - shi, so also 0 < j < ny,
  // and the +y neighbour j0 + TY stays <= ny. Interior pairs: the lane nodes
  // i0 = xs - 2 .. i0 + 63 and the +x neighbour i0 + 64 satisfy the same in
  // x; xs is even (i0 = xb0 - 2 the first even node above slo).
  const int nby = (c->ny + 1 + TY - 2) / (TY - 1);
  A.nbx = (c->nx + 1 + kEmTX - 2) / (kEmTX - 1);
  A.iby0 = A.iby1 = 0;
  for (int b = 0; b < nby; ++b) {
    const int j0 = b * (TY - 1) - 1;
    if (j0 >= c->slo[1] + 1 && j0 + TY <= c->ny - c->shi[1]) {
      if (A.iby1 == 0) A.iby0 = b;
      A.iby1 = b + 1;
    }
  }
  A.xb0 = (c->slo[0] + 4) & ~1;  // smallest even xs with xs - 2 >= slo + 1
  A.npx = std::max(0, (c->nx - c->shi[0] - A.xb0) / 62);
  if (A.npx == 0 || A.iby1 == A.iby0) A.npx = A.iby0 = A.iby1 = 0;
  A.xb1 = A.xb0 + 62 * A.npx;
  A.nl = A.npx ? (A.xb0 + kEmTX - 2) / (kEmTX - 1) : 0;
  A.nr = A.npx ? (c->nx + 1 - A.xb1 + kEmTX - 2) / (kEmTX - 1) : 0;
  A.n_border = (nby - (A.iby1 - A.iby0)) * A.nbx + (A.iby1 - A.iby0) * (A.nl + A.nr);
  A.dt = (R)c->dt;
  A.src_row = c->src_row;
  A.src_ent = c->src_ent;
  A.src_amp = (const R *)c->src_amp;
  A.amp_len = c->amp_len;
  A.Qs = accum ? (R *)c->Qs : nullptr;
  A.Q = c->Q;
  A.tmQ = c->tmQ[t];
  A.tmV = c->tmV[t];
  A.tmQ2 = c->tmQ2[t];
  A.tmV2 = c->tmV2[t];
  A.zt = (const R *)c->zt;
  A.err = c->dev_err;
  A.wait = c->wait_cycles;
  return A;
}

// The arguments of one step: the E/H buffers read (parity o) and written,
// their descriptors, the source time offset s within the call, the step's
// Joule window position (-1: not accumulating).
template <typename R, int TY>
static void em_args_step(cosim_ctx *c, EmArgs<R> &A, int o, int s, int fold) {
  constexpr int t = em_ty_index(TY);
  const int n = o ^ 1;
  for (int a = 0; a < 3; ++a) {
    A.Eo[a] = (const R *)c->E[o][a];
    A.En[a] = (R *)c->E[n][a];
    A.Ho[a] = (const R *)c->H[o][a];
    A.Hn[a] = (R *)c->H[n][a];
    for (int s2 = 0; s2 < 2; ++s2) {
      A.xEo[a][s2] = (const R *)c->xE[o][a][s2];
      A.dEo[a][s2] = (const R *)c->dE[o][a][s2];
      A.xEn[a][s2] = (R *)c->xE[n][a][s2];
      A.dEn[a][s2] = (R *)c->dE[n][a][s2];
      A.xHo[a][s2] = (const R *)c->xH[o][a][s2];
      A.dHo[a][s2] = (const R *)c->dH[o][a][s2];
      A.xHn[a][s2] = (R *)c->xH[n][a][s2];
      A.dHn[a][s2] = (R *)c->dH[n][a][s2];
      A.lEo[a][s2] = (const R *)c->lE[o][a][s2];
      A.lEn[a][s2] = (R *)c->lE[n][a][s2];
      A.lHo[a][s2] = (const R *)c->lH[o][a][s2];
      A.lHn[a][s2] = (R *)c->lH[n][a][s2];
    }
    A.tmE[a] = c->tmE[t][o][a];
    A.tmE2[a] = c->tmE2[t][o][a];
    A.tmH2[a] = c->tmH2[t][o][a];
    A.tmH[a] = c->tmH[t][o][a];
  }
  A.step_base = c->dstep;
  A.step_off = s;
  A.fold = fold;
}

template <typename R, int TY>
static cosim_status em_steps_tile(cosim_ctx *c, int64_t nsteps, bool accum, bool coupled, bool fused = false,
                                  bool probe = false) {
  EmArgs<R> A = em_args_base<R, TY>(c, accum);
  const dim3 blk(kEmTX, TY);
  const dim3 grd(A.n_border + A.npx * (A.iby1 - A.iby0));
  const size_t smem = em_smem_bytes<R, TY>((int)c->mats.size());
  constexpr int t = em_ty_index(TY);
  for (int64_t s = 0; s < nsteps; ++s) {
    // the step's position in the Joule window: each node plane folds once per
    // window, the planes spread over its steps
    em_args_step<R, TY>(c, A, c->par, (int)s, accum ? (int)(c->n_acc % kJouleWindow) : -1);
    A.tmT = c->tmT[t][c->tpar];
    A.tmT2 = c->tmT2[t][c->tpar];
    A.Pout = (R *)c->P;
    A.inv_dt = (R)(1.0 / c->dt);
    A.Tth = (R *)c->T[c->tpar ^ 1];
    A.T_amb = (R)(c->T_amb - c->T_init);
    for (int f = 0; f < 6; ++f) A.hconv[f] = (R)c->h_conv[f];
    // peak tracking (cosim_coupled_march): the step's maximum rise on check steps
    A.peak = (coupled && c->pk_check_every > 0 &&
              ((c->step + 1 - c->pk_base) % c->pk_check_every == 0 || s == nsteps - 1))
                 ? c->pk
                 : nullptr;
    const bool small = c->npad < (1LL << 31);
    if constexpr (TY == kEmTY) {
      if (coupled && fused)
        small ? launch_em<R, int, TY, true, true>(grd, blk, smem, c->stream, A)
              : launch_em<R, long long, TY, true, true>(grd, blk, smem, c->stream, A);
      else if (coupled)
        small ? launch_em<R, int, TY, true>(grd, blk, smem, c->stream, A)
              : launch_em<R, long long, TY, true>(grd, blk, smem, c->stream, A);
      else
        small ? launch_em<R, int, TY, false>(grd, blk, smem, c->stream, A)
              : launch_em<R, long long, TY, false>(grd, blk, smem, c->stream, A);
    } else {  // the small tile exists for FP32 plain steps only
      small ? launch_em<R, int, TY, false>(grd, blk, smem, c->stream, A)
            : launch_em<R, long long, TY, false>(grd, blk, smem, c->stream, A);
    }
    CHECK_LAUNCH(c);
    if (probe) continue;
    ++c->launches;
    // coupled: the launch also took the thermal step T^{n+1} = T^n + dt/C
    // (-M_kk T^n + P^{n+1}) with the EM dt (Eq. 5) into the other buffer
    if (coupled) {
      if (!fused) {  // the thermal step as its own launch (tracking the step's maximum on check steps)
        const cosim_status ts = launch_thermal<R>(c, (R)c->dt, true, A.peak);
        if (ts != COSIM_OK) return ts;
      }
      c->tpar ^= 1;
      if (A.peak != nullptr) {  // a check step: compare with the recorded peak, copy T if higher
        peak_check_kernel<<<1, 1, 0, c->stream>>>(c->pk, c->step + 1); ++c->launches;
        peak_snapshot_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(c->npad, c->pk, (const R *)c->T[c->tpar],
                                                                   (R *)c->T_peak); ++c->launches;
        CHECK_LAUNCH(c);
      }
    }
    c->par ^= 1;
    c->step++;
    if (accum) {
      c->n_acc++;
      c->qs_dirty = true;  // some planes hold energy of their current window
    }
  }
  if (nsteps > 0 && !probe) {
    step_advance_kernel<<<1, 1, 0, c->stream>>>(c->dstep, nsteps);
    ++c->launches;
    CHECK_LAUNCH(c);
  }
  return COSIM_OK;
}

template <typename R>
static cosim_status em_steps_t(cosim_ctx *c, int64_t nsteps, bool accum, bool coupled, bool fused) {
  if constexpr (sizeof(R) == 4)
    if (!coupled && c->em_ty == kEmTYSmall) return em_steps_tile<R, kEmTYSmall>(c, nsteps, accum, false);
  return em_steps_tile<R, kEmTY>(c, nsteps, accum, coupled, coupled && fused);
}

static cosim_status em_steps_any(cosim_ctx *c, int64_t nsteps, bool acc, bool coupled, bool fused = false) {
  // groups of at most 2^30 steps keep the per-launch offset an int
  while (nsteps > 0) {
    const int64_t n = std::min<int64_t>(nsteps, 1LL << 30);
    const cosim_status st =
        c->prec == COSIM_FP64 ? em_steps_t<double>(c, n, acc, coupled, fused) : em_steps_t<float>(c, n, acc, coupled, fused);
    if (st != COSIM_OK) return st;
    nsteps -= n;
  }
  return COSIM_OK;
}

extern "C" cosim_status cosim_em_steps(cosim_ctx *c, int64_t nsteps, uint32_t flags) {
  if (!c) return COSIM_ERR_INVALID;
  if (nsteps < 0 || (flags & ~kEmFlags)) return fail(c, COSIM_ERR_INVALID, "bad nsteps or flags");
  return em_steps_any(c, nsteps, flags & COSIM_ACCUM_JOULE, flags & (COSIM_COUPLED_THERMAL | COSIM_COUPLED_FUSED),
                      flags & COSIM_COUPLED_FUSED);
}

static cosim_status check_device_wait(cosim_ctx *c);

// image -> value of ordered_bits (host side)
static double from_ordered(unsigned long long b) {
  b = (b >> 63) ? (b & ~(1ull << 63)) : ~b;
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}

extern "C" cosim_status cosim_coupled_march(cosim_ctx *c, int64_t nsteps, uint32_t flags, int64_t check_every,
                                            int32_t reset, cosim_peak_report *rep) {
  if (!c) return COSIM_ERR_INVALID;
  if (nsteps < 0 || check_every <= 0) return fail(c, COSIM_ERR_INVALID, "nsteps < 0 or check_every <= 0");
  if (flags & ~kEmFlags) return fail(c, COSIM_ERR_INVALID, "unknown flags");
  if (!c->pk) {
    ALLOC(c, c->pk, 5 * sizeof(unsigned long long));
    ALLOC(c, c->T_peak, c->npad * c->rsz);
    reset = 1;
  }
  if (reset) {
    CHECK_CUDA(c, cudaMemsetAsync(c->pk, 0, 5 * sizeof(unsigned long long), c->stream));
    CHECK_CUDA(c, cudaMemcpyAsync(c->T_peak, c->T[c->tpar], c->npad * c->rsz, cudaMemcpyDeviceToDevice, c->stream));
  }
  c->pk_check_every = check_every;
  c->pk_base = c->step;
  cosim_status st = em_steps_any(c, nsteps, (flags & COSIM_ACCUM_JOULE) != 0, true, (flags & COSIM_COUPLED_FUSED) != 0);
  c->pk_check_every = 0;
  if (st != COSIM_OK) return st;
  if (rep) {
    unsigned long long h[5];
    CHECK_CUDA(c, cudaMemcpyAsync(h, c->pk, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if ((st = check_device_wait(c)) != COSIM_OK) return st;
    rep->peaks = (int64_t)h[3];
    rep->step = h[3] ? (int64_t)h[4] : -1;
    rep->T_max = h[3] ? from_ordered(h[1]) + c->T_init : c->T_init;
  }
  return COSIM_OK;
}

static void drop_graph(cosim_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_nsteps = 0;
}

extern "C" cosim_status cosim_em_graph_capture(cosim_ctx *c, int64_t nsteps, uint32_t flags) {
  if (!c) return COSIM_ERR_INVALID;
  if (nsteps <= 0 || nsteps % kJouleWindow != 0 || nsteps > (1LL << 30) ||
      (flags & ~kEmFlags))
    return fail(c, COSIM_ERR_INVALID, "graph steps must be a positive multiple of 32 (the Joule window), <= 2^30");
  if (c->stream == nullptr) return fail(c, COSIM_ERR_INVALID, "graph capture needs a non-default stream");
  const bool acc = flags & COSIM_ACCUM_JOULE;
  if (acc && c->n_acc % kJouleWindow != 0)
    return fail(c, COSIM_ERR_INVALID, "capture with Joule accumulation must start on a 32-step window boundary");
  drop_graph(c);
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  // capturing records the launches without running them: keep the host
  // bookkeeping as it was and apply it per replay instead
  const long long step = c->step, n_acc = c->n_acc, launches = c->launches;
  const int par = c->par;
  const bool dirty = c->qs_dirty;
  CHECK_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const bool cpl = flags & (COSIM_COUPLED_THERMAL | COSIM_COUPLED_FUSED);
  const int tpar = c->tpar;
  cosim_status st = em_steps_any(c, nsteps, acc, cpl, (flags & COSIM_COUPLED_FUSED) != 0);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  const long long captured = c->launches - launches;
  c->step = step, c->n_acc = n_acc, c->launches = launches, c->par = par, c->qs_dirty = dirty, c->tpar = tpar;
  if (st != COSIM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess || graph == nullptr) {
    cudaGetLastError();
    return fail(c, COSIM_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    c->gexec = nullptr;
    cudaGetLastError();
    return fail(c, COSIM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  }
  c->g_nsteps = nsteps;
  c->g_accum = acc;
  c->g_coupled = cpl;
  c->g_par = par;
  c->g_tpar = tpar;
  c->g_launches = captured;
  return COSIM_OK;
}

extern "C" cosim_status cosim_em_graph_launch(cosim_ctx *c, int64_t count) {
  if (!c) return COSIM_ERR_INVALID;
  if (count < 0) return fail(c, COSIM_ERR_INVALID, "bad count");
  if (!c->gexec) return fail(c, COSIM_ERR_INVALID, "no captured EM graph");
  if (c->par != c->g_par) return fail(c, COSIM_ERR_INVALID, "the E/H parity differs from the captured one");
  if (c->g_coupled && c->tpar != c->g_tpar)
    return fail(c, COSIM_ERR_INVALID, "the temperature buffer parity differs from the captured one");
  if (c->g_accum && c->n_acc % kJouleWindow != 0)
    return fail(c, COSIM_ERR_INVALID, "Joule window position differs from the captured one");
  for (int64_t r = 0; r < count; ++r) {
    CHECK_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    c->step += c->g_nsteps;
    c->launches += c->g_launches;
    if (c->g_accum) {
      c->n_acc += c->g_nsteps;
      c->qs_dirty = true;
    }
  }
  return COSIM_OK;
}

// ---------------------------------------------------------------- design batches

struct cosim_batch {
  std::vector<cosim_ctx *> ctx;  // in tile order: the contexts with the most nodes first
  std::vector<long long> src_version;
  int prec = COSIM_FP32;
  cudaStream_t stream = nullptr;
  bool persistent = false;
  // groups of up to kBatchMax consecutive contexts, one launch each per step
  struct Group {
    int first = 0, n = 0, total = 0, grid = 0;
    bool wide = false;               // some context needs 64-bit node offsets
    size_t smem = 0;
    std::vector<unsigned char> args;  // EmBatchArgs<R>[4]: [accum][parity] (the fold is a launch parameter)
  };
  std::vector<Group> groups;
  unsigned *work = nullptr;      // two tile counters per group (persistent launches)
  long long **dsteps = nullptr;  // the contexts' device source time counters
  long long n_launch = 0;        // persistent steps so far (which counter is next)
  cudaGraphExec_t gexec = nullptr;
  int64_t g_nsteps = 0;
  bool g_accum = false;
  int g_par = 0;
  long long g_launches = 0;
  std::string err;
};

static cosim_status bfail(cosim_batch *b, cosim_status s, const std::string &m) {
  b->err = m;
  return s;
}
#define BCHECK(b, call)                                                       \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      (b)->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return COSIM_ERR_CUDA;                                                  \
    }                                                                         \
  } while (0)

// advance every context's device source time counter after a group of steps
__global__ void batch_step_advance_kernel(long long *const *steps, int n, long long nsteps) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < n) *steps[d] += nsteps;
}

template <typename R>
static cosim_status batch_build(cosim_batch *b) {
  const int n = (int)b->ctx.size();
  std::vector<long long *> st(n);
  int dev = 0, nsm = 0;
  BCHECK(b, cudaGetDevice(&dev));
  BCHECK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  for (int first = 0; first < n; first += kBatchMax) {
    cosim_batch::Group g;
    g.first = first;
    g.n = std::min(kBatchMax, n - first);
    g.args.assign(4 * sizeof(EmBatchArgs<R>), 0);
    EmBatchArgs<R> *P = reinterpret_cast<EmBatchArgs<R> *>(g.args.data());
    for (int d = 0; d < g.n; ++d) {
      cosim_ctx *c = b->ctx[first + d];
      for (int acc = 0; acc < 2; ++acc) {
        const EmArgs<R> base = em_args_base<R, kEmTY>(c, acc != 0);
        for (int o = 0; o < 2; ++o) {
          EmArgs<R> A = base;
          em_args_step<R, kEmTY>(c, A, o, 0, -1);
          P[2 * acc + o].a[d] = A;
        }
      }
      const EmArgs<R> &A = P[0].a[d];
      const int tiles = A.n_border + A.npx * (A.iby1 - A.iby0);
      for (int v = 0; v < 4; ++v) P[v].cta_start[d + 1] = P[v].cta_start[d] + tiles;
      st[first + d] = c->dstep;
      g.smem = std::max(g.smem, em_smem_bytes<R, kEmTY>((int)c->mats.size()));
      g.wide = g.wide || c->npad >= (1LL << 31);
    }
    for (int v = 0; v < 4; ++v) P[v].n = g.n;
    g.total = P[0].cta_start[g.n];
    g.grid = g.total;
    if (b->persistent) {  // about the CTAs that are resident at once
      int occ = 0;
      BCHECK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &occ, g.wide ? (const void *)em_batch_kernel<R, long long, kEmTX, kEmTY>
                                 : (const void *)em_batch_kernel<R, int, kEmTX, kEmTY>,
                    kEmTX * kEmTY, g.smem));
      g.grid = std::max(1, std::min(g.total, nsm * std::max(occ, 1)));
    }
    b->groups.push_back(std::move(g));
  }
  BCHECK(b, cudaMalloc((void **)&b->work, 2 * b->groups.size() * sizeof(unsigned)));
  BCHECK(b, cudaMalloc((void **)&b->dsteps, n * sizeof(long long *)));
  BCHECK(b, cudaMemset(b->work, 0, 2 * b->groups.size() * sizeof(unsigned)));
  BCHECK(b, cudaMemcpy(b->dsteps, st.data(), n * sizeof(long long *), cudaMemcpyHostToDevice));
  return COSIM_OK;
}

extern "C" cosim_status cosim_batch_create(cosim_ctx *const *ctxs, int32_t n, int32_t persistent,
                                           cosim_batch **out) {
  if (!out) return COSIM_ERR_INVALID;
  *out = nullptr;
  if (!ctxs || n < 1) return COSIM_ERR_INVALID;
  cosim_batch *b = new cosim_batch();
  std::vector<std::pair<int, cosim_ctx *>> order;
  for (int d = 0; d < n; ++d) {
    cosim_ctx *c = ctxs[d];
    if (!c || c->prec != ctxs[0]->prec || c->stream != ctxs[0]->stream) {
      delete b;
      return COSIM_ERR_INVALID;
    }
    for (int q = 0; q < d; ++q)
      if (ctxs[q] == c) {
        delete b;
        return COSIM_ERR_INVALID;
      }
    order.emplace_back(-(int)((long long)(c->nx + 1) * (c->ny + 1) * (c->nz + 1) / 1024), c);
  }
  // the largest designs first: in a persistent launch their tiles are taken
  // first and the small designs' tiles fill the tail
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<int, cosim_ctx *> &a, const std::pair<int, cosim_ctx *> &b2) {
                     return a.first < b2.first;
                   });
  for (auto &pc : order) {
    b->ctx.push_back(pc.second);
    b->src_version.push_back(pc.second->src_version);
  }
  b->prec = ctxs[0]->prec;
  b->stream = ctxs[0]->stream;
  b->persistent = persistent != 0;
  const cosim_status st = b->prec == COSIM_FP64 ? batch_build<double>(b) : batch_build<float>(b);
  if (st != COSIM_OK) {
    g_create_error = b->err;
    cosim_batch_destroy(b);
    return st;
  }
  *out = b;
  return COSIM_OK;
}

// the contexts must step together: same E/H parity, same Joule window
// position, sources unchanged since the batch was built
static cosim_status batch_check(cosim_batch *b, bool accum) {
  cosim_ctx *c0 = b->ctx[0];
  for (size_t d = 0; d < b->ctx.size(); ++d) {
    cosim_ctx *c = b->ctx[d];
    if (c->src_version != b->src_version[d])
      return bfail(b, COSIM_ERR_INVALID, "a context's sources changed after the batch was created");
    if (c->par != c0->par || (accum && c->n_acc % kJouleWindow != c0->n_acc % kJouleWindow))
      return bfail(b, COSIM_ERR_INVALID, "the contexts are at different E/H parities or Joule window positions");
  }
  return COSIM_OK;
}

template <typename R>
static cosim_status batch_steps_t(cosim_batch *b, int64_t nsteps, bool accum) {
  const int n = (int)b->ctx.size();
  cosim_ctx *c0 = b->ctx[0];
  const dim3 blk(kEmTX, kEmTY);
  for (int64_t s = 0; s < nsteps; ++s) {
    const int fold = accum ? (int)(c0->n_acc % kJouleWindow) : -1;  // window position (the kernel parameter)
    const int variant = 2 * (accum ? 1 : 0) + c0->par;
    const int cnt = (int)(b->n_launch & 1);
    if (b->persistent) ++b->n_launch;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      const cosim_batch::Group &g = b->groups[gi];
      const EmBatchArgs<R> &P = reinterpret_cast<const EmBatchArgs<R> *>(g.args.data())[variant];
      unsigned *w = b->persistent ? b->work + 2 * gi + cnt : nullptr;
      unsigned *wn = b->persistent ? b->work + 2 * gi + (cnt ^ 1) : nullptr;
      if (g.wide)
        em_batch_kernel<R, long long, kEmTX, kEmTY><<<g.grid, blk, g.smem, b->stream>>>(P, (int)s, fold, w, wn);
      else
        em_batch_kernel<R, int, kEmTX, kEmTY><<<g.grid, blk, g.smem, b->stream>>>(P, (int)s, fold, w, wn);
      BCHECK(b, cudaGetLastError());
    }
    for (cosim_ctx *c : b->ctx) {
      c->par ^= 1;
      c->step++;
      if (accum) {
        c->n_acc++;
        c->qs_dirty = true;
      }
    }
    c0->launches += (long long)b->groups.size();
  }
  if (nsteps > 0) {
    batch_step_advance_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->dsteps, n, nsteps);
    BCHECK(b, cudaGetLastError());
    ++c0->launches;
  }
  return COSIM_OK;
}

static cosim_status batch_steps(cosim_batch *b, int64_t nsteps, bool accum) {
  while (nsteps > 0) {  // groups of at most 2^30 steps keep the step offset an int
    const int64_t q = std::min<int64_t>(nsteps, 1LL << 30);
    const cosim_status st = b->prec == COSIM_FP64 ? batch_steps_t<double>(b, q, accum) : batch_steps_t<float>(b, q, accum);
    if (st != COSIM_OK) return st;
    nsteps -= q;
  }
  return COSIM_OK;
}

extern "C" cosim_status cosim_batch_em_steps(cosim_batch *b, int64_t nsteps, uint32_t flags) {
  if (!b) return COSIM_ERR_INVALID;
  if (nsteps < 0 || (flags & ~COSIM_ACCUM_JOULE)) return bfail(b, COSIM_ERR_INVALID, "bad nsteps or flags");
  const bool acc = flags & COSIM_ACCUM_JOULE;
  const cosim_status st = batch_check(b, acc);
  if (st != COSIM_OK) return st;
  for (cosim_ctx *c : b->ctx) drop_graph(c);  // (a context's own graph assumes its own step sequence)
  return batch_steps(b, nsteps, acc);
}

static void batch_drop_graph(cosim_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_nsteps = 0;
}

extern "C" cosim_status cosim_batch_graph_capture(cosim_batch *b, int64_t nsteps, uint32_t flags) {
  if (!b) return COSIM_ERR_INVALID;
  if (nsteps <= 0 || nsteps % kJouleWindow != 0 || nsteps > (1LL << 30) || (flags & ~COSIM_ACCUM_JOULE))
    return bfail(b, COSIM_ERR_INVALID, "graph steps must be a positive multiple of 32 (the Joule window), <= 2^30");
  if (b->stream == nullptr) return bfail(b, COSIM_ERR_INVALID, "graph capture needs a non-default stream");
  const bool acc = flags & COSIM_ACCUM_JOULE;
  cosim_status st = batch_check(b, acc);
  if (st != COSIM_OK) return st;
  if (acc && b->ctx[0]->n_acc % kJouleWindow != 0)
    return bfail(b, COSIM_ERR_INVALID, "capture with Joule accumulation must start on a 32-step window boundary");
  batch_drop_graph(b);
  BCHECK(b, cudaStreamSynchronize(b->stream));
  // capturing records the launches without running them: the contexts'
  // bookkeeping is restored afterwards and applied per replay
  struct Saved { long long step, n_acc, launches; int par; bool dirty; };
  std::vector<Saved> sv;
  for (cosim_ctx *c : b->ctx) sv.push_back({c->step, c->n_acc, c->launches, c->par, c->qs_dirty});
  const long long nl = b->n_launch, l0 = b->ctx[0]->launches;
  BCHECK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  st = batch_steps(b, nsteps, acc);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  const long long captured = b->ctx[0]->launches - l0;
  for (size_t d = 0; d < b->ctx.size(); ++d) {
    cosim_ctx *c = b->ctx[d];
    c->step = sv[d].step, c->n_acc = sv[d].n_acc, c->launches = sv[d].launches, c->par = sv[d].par;
    c->qs_dirty = sv[d].dirty;
  }
  b->n_launch = nl;
  if (st != COSIM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess || graph == nullptr) {
    cudaGetLastError();
    return bfail(b, COSIM_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->gexec = nullptr;
    cudaGetLastError();
    return bfail(b, COSIM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  }
  b->g_nsteps = nsteps;
  b->g_accum = acc;
  b->g_par = b->ctx[0]->par;
  b->g_launches = captured;
  return COSIM_OK;
}

extern "C" cosim_status cosim_batch_graph_launch(cosim_batch *b, int64_t count) {
  if (!b) return COSIM_ERR_INVALID;
  if (!b->gexec) return bfail(b, COSIM_ERR_INVALID, "no captured graph");
  if (count < 0) return bfail(b, COSIM_ERR_INVALID, "count < 0");
  cosim_status st = batch_check(b, b->g_accum);
  if (st != COSIM_OK) return st;
  if (b->ctx[0]->par != b->g_par || (b->g_accum && b->ctx[0]->n_acc % kJouleWindow != 0))
    return bfail(b, COSIM_ERR_INVALID, "the contexts' parity or Joule window differs from the captured one");
  for (int64_t q = 0; q < count; ++q) {
    BCHECK(b, cudaGraphLaunch(b->gexec, b->stream));
    for (cosim_ctx *c : b->ctx) {
      c->step += b->g_nsteps;
      if (b->g_accum) {
        c->n_acc += b->g_nsteps;
        c->qs_dirty = true;
      }
    }
    b->ctx[0]->launches += b->g_launches;
  }
  return COSIM_OK;
}

extern "C" const char *cosim_batch_last_error(const cosim_batch *b) { return b ? b->err.c_str() : g_create_error.c_str(); }

extern "C" void cosim_batch_destroy(cosim_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  cudaFree(b->work);
  cudaFree(b->dsteps);
  delete b;
}

// move the short-window Joule energy into the FP64 total (Q += Qs, Qs = 0)
template <typename R>
__global__ void __launch_bounds__(256) joule_flush_kernel(long long n, double *Q, R *Qs) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const R v = Qs[q];
    if (v != R(0)) {
      Q[q] += (double)v;
      Qs[q] = R(0);
    }
  }
}

// op 1 of the finalisation as one streaming pass over the padded node arrays:
// P = (Q + Qs) * inv_t, the burst-averaged power per node, with the pending
// short-window energy Qs added on the fly (Qs null: none pending); Q and Qs
// are left as they are. FP32 contexts form P in FP32 (Q rounded to FP32
// first, then one addition and one multiplication; P is stored in FP32
// anyway): FP64 arithmetic is slow on this part, and one FP64 multiplication
// per node bound this pass. FP32 contexts stream four nodes per access (n is
// a multiple of 4; the padding gives 0).
template <typename R>
__global__ void __launch_bounds__(256) joule_power_kernel(long long n, const double *Q, const R *Qs, R *P,
                                                          double inv_t) {
  const long long stride = (long long)gridDim.x * blockDim.x, first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    const float it = (float)inv_t;
    for (long long v = first; v < (n >> 2); v += stride) {
      const float4 w = Qs != nullptr ? reinterpret_cast<const float4 *>(Qs)[v] : make_float4(0.f, 0.f, 0.f, 0.f);
      const double2 q01 = reinterpret_cast<const double2 *>(Q)[2 * v], q23 = reinterpret_cast<const double2 *>(Q)[2 * v + 1];
      reinterpret_cast<float4 *>(P)[v] =
          make_float4(((float)q01.x + w.x) * it, ((float)q01.y + w.y) * it, ((float)q23.x + w.z) * it,
                      ((float)q23.y + w.w) * it);
    }
  } else {
    for (long long q = first; q < n; q += stride) P[q] = (Q[q] + (Qs != nullptr ? Qs[q] : R(0))) * inv_t;
  }
}

static cosim_status joule_flush(cosim_ctx *c) {
  if (!c->qs_dirty) return COSIM_OK;
  if (c->prec == COSIM_FP64)
    joule_flush_kernel<double><<<kRedBlocks, 256, 0, c->stream>>>(c->npad, c->Q, (double *)c->Qs);
  else
    joule_flush_kernel<float><<<kRedBlocks, 256, 0, c->stream>>>(c->npad, c->Q, (float *)c->Qs);
  ++c->launches;
  CHECK_LAUNCH(c);
  c->qs_dirty = false;
  return COSIM_OK;
}

// ---------------------------------------------------------------- reductions

static cosim_status sum_q(cosim_ctx *c, double *out) {
  sum_partial_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->npad, c->Q, c->part); ++c->launches;
  CHECK_LAUNCH(c);
  reduce_final_kernel<<<1, 1024, 0, c->stream>>>(c->part, kRedBlocks, c->scal); ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, c->scal, 8, cudaMemcpyDeviceToHost, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = c->host_scal[0];
  return COSIM_OK;
}

template <typename R>
static cosim_status joule_t(cosim_ctx *c, int op) {
  const dim3 blk(32, 8), grd((c->nx + 1 + 31) / 32, (c->ny + 1 + 7) / 8);
  const size_t smem = c->mats.size() * M_COLS * sizeof(R);
  const double inv_t = c->n_acc > 0 ? 1.0 / (c->n_acc * c->dt) : 0.0;
  if (op == COSIM_JOULE_FINALIZE_AVG_POWER) {  // the pending window added on the fly, not folded
    joule_power_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(c->npad, c->Q, c->qs_dirty ? (const R *)c->Qs : nullptr,
                                                             (R *)c->P, inv_t); ++c->launches;
    CHECK_LAUNCH(c);
    return COSIM_OK;
  }
  {
    cosim_status fs = joule_flush(c);
    if (fs != COSIM_OK) return fs;
  }
  joule_finalize_kernel<R><<<grd, blk, smem, c->stream>>>(make_geo<R>(c), c->Q, (R *)c->P, (R *)c->T[c->tpar],
                                                          inv_t, op); ++c->launches;
  CHECK_LAUNCH(c);
  return COSIM_OK;
}

extern "C" cosim_status cosim_joule_accumulate(cosim_ctx *c, int32_t op, double *total) {
  if (!c) return COSIM_ERR_INVALID;
  if (op < 0 || op > 2) return fail(c, COSIM_ERR_INVALID, "bad joule op");
  if (op == COSIM_JOULE_RESET) {
    if (total) *total = 0;
    CHECK_CUDA(c, cudaMemsetAsync(c->Q, 0, c->npad * 8, c->stream));
    CHECK_CUDA(c, cudaMemsetAsync(c->Qs, 0, c->npad * c->rsz, c->stream));
    c->qs_dirty = false;
    c->n_acc = 0;
    return COSIM_OK;
  }
  cosim_status st = c->prec == COSIM_FP64 ? joule_t<double>(c, op) : joule_t<float>(c, op);
  if (st != COSIM_OK) return st;
  if (total) {
    if ((st = joule_flush(c)) != COSIM_OK) return st;  // the total sums Q only
    st = sum_q(c, total);
    if (st != COSIM_OK) return st;
    if (!std::isfinite(*total)) return fail(c, COSIM_ERR_NONFINITE, "non-finite Joule energy");
  }
  return COSIM_OK;
}

// ---------------------------------------------------------------- thermal

template <typename R>
static ThArgs<R> th_args(cosim_ctx *c) {
  ThArgs<R> A;
  A.g = make_geo<R>(c);
  A.To = (const R *)c->T[c->tpar];
  A.Tn = (R *)c->T[c->tpar ^ 1];
  A.P = (const R *)c->P;
  A.zt = (const R *)c->zt;
  A.T_amb = (R)(c->T_amb - c->T_init);
  for (int f = 0; f < 6; ++f) A.hconv[f] = (R)c->h_conv[f];
  A.ratio_out = nullptr;
  A.dt = 0;
  return A;
}

template <typename R>
static cosim_status thermal_limit_t(cosim_ctx *c) {
  ThArgs<R> A = th_args<R>(c);
  A.ratio_out = (R *)c->scratch;
  const dim3 blk(32, 8), grd((c->nx + 1 + 31) / 32, (c->ny + 1 + 7) / 8);
  const size_t smem = (c->mats.size() + 1) * sizeof(typename Pair2<R>::T);
  thermal_kernel<R, 1><<<grd, blk, smem, c->stream>>>(A); ++c->launches;
  CHECK_LAUNCH(c);
  min_partial_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(A.g, (const R *)c->scratch, c->part); ++c->launches;
  CHECK_LAUNCH(c);
  min_final_kernel<<<1, 256, 0, c->stream>>>(c->part, kRedBlocks, c->scal); ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, c->scal, 8, cudaMemcpyDeviceToHost, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  c->dt_th_limit = c->host_scal[0];
  return COSIM_OK;
}

static cosim_status ensure_th_limit(cosim_ctx *c) {
  if (c->dt_th_limit > 0) return COSIM_OK;
  return c->prec == COSIM_FP64 ? thermal_limit_t<double>(c) : thermal_limit_t<float>(c);
}

template <typename R>
static cosim_status thermal_steps_t(cosim_ctx *c, int64_t nsteps, double dt) {
  for (int64_t s = 0; s < nsteps; ++s) {
    const cosim_status st = launch_thermal<R>(c, (R)dt);
    if (st != COSIM_OK) return st;
    c->tpar ^= 1;
  }
  return COSIM_OK;
}

extern "C" cosim_status cosim_thermal_steps(cosim_ctx *c, int64_t nsteps, double dt) {
  if (!c) return COSIM_ERR_INVALID;
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, COSIM_ERR_INVALID, "bad thermal step arguments");
  if (dt <= 0) {
    cosim_status st = ensure_th_limit(c);
    if (st != COSIM_OK) return st;
    dt = c->thermal_safety * c->dt_th_limit;
  }
  return c->prec == COSIM_FP64 ? thermal_steps_t<double>(c, nsteps, dt) : thermal_steps_t<float>(c, nsteps, dt);
}

// ---------------------------------------------------------------- mechanics

static cosim_status mech_alloc(cosim_ctx *c) {
  if (c->mech_ready) return COSIM_OK;
  ALLOC(c, c->mask, c->npad);
  for (int a = 0; a < 3; ++a) {
    ALLOC(c, c->U[a], c->npad * c->rsz);
    ALLOC(c, c->F[a], c->npad * c->rsz);
    ALLOC(c, c->Rv[a], c->npad * c->rsz);
    ALLOC(c, c->Pv[a], c->npad * c->rsz);
    ALLOC(c, c->Pv2[a], c->npad * c->rsz);
    ALLOC(c, c->Qv[a], c->npad * c->rsz);
    ALLOC(c, c->Dinv[a], c->npad * c->rsz);
  }
  ALLOC(c, c->VM, (size_t)c->nx * c->ny * c->nz * c->rsz);
  ALLOC(c, c->UMAG, c->npad * c->rsz);
  ALLOC(c, c->cg, sizeof(CgScalars));
  cosim_status st;
  for (int a = 0; a < 3; ++a)
    if ((st = encode_node_map(c, &c->mvU[0][a], c->Pv[a], kMvTY + 1, kMvElems + 4)) != COSIM_OK ||
        (st = encode_node_map(c, &c->mvU[1][a], c->Pv2[a], kMvTY + 1, kMvElems + 4)) != COSIM_OK ||
        (st = encode_node_map(c, &c->mvR[a], c->Rv[a], kMvTY + 1, kMvElems + 4)) != COSIM_OK ||
        (st = encode_node_map(c, &c->mvD[a], c->Dinv[a], kMvTY + 1, kMvElems + 4)) != COSIM_OK)
      return st;
  {
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx + 1, (cuuint64_t)c->ny + 1, (cuuint64_t)c->nz + 1};
    const cuuint64_t strides[2] = {(cuuint64_t)c->px, (cuuint64_t)c->plane};
    const cuuint32_t box[3] = {(cuuint32_t)kMvElems + 16, (cuuint32_t)kMvTY + 1, 1};
    if ((st = encode_map(c, &c->mvM, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, c->mask, dims, strides, box)) != COSIM_OK)
      return st;
  }
  if ((st = encode_voxel_map(c, &c->mvV, kMvTY, kMvElems + 16)) != COSIM_OK) return st;
  c->mech_ready = true;
  return COSIM_OK;
}

static cosim_status upload_mask(cosim_ctx *c, const cosim_stress_opts *o) {
  if (o->bc < 0 || o->bc > 2) return fail(c, COSIM_ERR_INVALID, "bad mechanical support");
  if (o->bc == COSIM_MECH_MASK && !o->node_mask) return fail(c, COSIM_ERR_INVALID, "node_mask is NULL");
  if (o->bc != COSIM_MECH_MASK) {  // built-in supports: written on the device, no host round trip
    CHECK_CUDA(c, cudaMemsetAsync(c->mask, 0, c->npad, c->stream));
    const int nb = o->bc == COSIM_MECH_CLAMPED_BOTTOM ? (int)std::min<long long>(
                                                            ((long long)(c->nx + 1) * (c->ny + 1) + 255) / 256, 4096)
                                                      : 1;
    support_mask_kernel<<<nb, 256, 0, c->stream>>>(c->mask, c->nx, c->ny, c->px, o->bc); ++c->launches;
    CHECK_LAUNCH(c);
    return COSIM_OK;
  }
  std::vector<uint8_t> m(c->npad, 0);
  for (int k = 0; k <= c->nz; ++k)
    for (int j = 0; j <= c->ny; ++j)
      for (int i = 0; i <= c->nx; ++i)
        m[(size_t)k * c->plane + (size_t)j * c->px + i] =
            o->node_mask[((size_t)k * (c->ny + 1) + j) * (c->nx + 1) + i] & 7;
  CHECK_CUDA(c, cudaMemcpyAsync(c->mask, m.data(), c->npad, cudaMemcpyHostToDevice, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return COSIM_OK;
}

template <typename R>
static cosim_status matvec_g(cosim_ctx *c, const Geo<R> &g, void *const u[3], void *const y[3], double *partial) {
  MvArgs<R> A;
  A.g = g;
  for (int a = 0; a < 3; ++a) {
    A.u[a] = (const R *)u[a];
    A.y[a] = (R *)y[a];
  }
  A.mask = c->mask;
  A.partial = partial;
  const dim3 blk(kMvTX, kMvTY);
  const dim3 grd((c->nx + 1 + kMvTX - 2) / (kMvTX - 1), (c->ny + 1 + kMvTY - 2) / (kMvTY - 1));
  // the CG direction buffers in the context precision have TMA descriptors: staged kernel
  const int buf = (u[0] == c->Pv[0] && u[1] == c->Pv[1] && u[2] == c->Pv[2])    ? 0
                  : (u[0] == c->Pv2[0] && u[1] == c->Pv2[1] && u[2] == c->Pv2[2]) ? 1
                                                                                  : -1;
  if (sizeof(R) == (size_t)c->rsz && buf >= 0) {
    MvTmaArgs<R> T{};
    T.a = A;
    for (int a = 0; a < 3; ++a) T.tmU[a] = c->mvU[buf][a];
    T.tmM = c->mvM;
    T.tmV = c->mvV;
    T.zt = (const R *)c->zt;
    T.err = c->dev_err;
  T.wait = c->wait_cycles;
    T.wait = c->wait_cycles;
    const size_t smem = mv_smem_bytes<R, kMvTY, false>((int)c->mats.size());
    const dim3 grd2((c->nx + 1 + kMvElems - 2) / (kMvElems - 1), (c->ny + 1 + kMvTY - 2) / (kMvTY - 1));
    hex8_matvec_tma_kernel<R, kMvTY, false><<<grd2, blk, smem, c->stream>>>(T); ++c->launches;
  } else {
    const size_t smem =
        ((size_t)c->mats.size() * M_COLS + 2 * 3 * (kMvTY + 1) * (kMvTX + 1) + 24 * kMvTY * kMvTX) * sizeof(R);
    hex8_matvec_kernel<R, kMvTX, kMvTY><<<grd, blk, smem, c->stream>>>(A); ++c->launches;
  }
  CHECK_LAUNCH(c);
  return COSIM_OK;
}

template <typename R>
static cosim_status matvec_t(cosim_ctx *c, void *const u[3], void *const y[3], double *partial) {
  return matvec_g<R>(c, make_geo<R>(c), u, y, partial);
}

// The PCG's fused direction update and product (hex8_matvec_tma_kernel, DIR):
// p_new = D^-1 r + beta p_old with p_old in direction buffer `from` (Pv or
// Pv2) and beta from the r.z pair of `parity`, written to the other buffer;
// U += alpha p_old with the previous iteration's alpha; Qv = K p_new with the
// p.Kp partial sums. Needs the DIR stages in shared memory (mv_dir_fits).
template <typename R>
static bool mv_dir_fits(const cosim_ctx *c) {
  return mv_smem_bytes<R, kMvTY, true>((int)c->mats.size()) <= kMaxSmemOptin;
}
template <typename R>
static cosim_status matvec_dir(cosim_ctx *c, int from, int parity, double *partial) {
  void *const *pnew = from ? c->Pv : c->Pv2;
  MvTmaArgs<R> T{};
  T.a.g = make_geo<R>(c);
  for (int a = 0; a < 3; ++a) {
    T.a.u[a] = (const R *)pnew[a];
    T.a.y[a] = (R *)c->Qv[a];
    T.tmU[a] = c->mvU[from][a];
    T.tmR[a] = c->mvR[a];
    T.tmD[a] = c->mvD[a];
    T.pn[a] = (R *)pnew[a];
    T.x[a] = (R *)c->U[a];  // the previous direction's step lands in the solution here
    T.po[a] = (const R *)(from ? c->Pv2 : c->Pv)[a];
  }
  T.a.mask = c->mask;
  T.a.partial = partial;
  T.tmM = c->mvM;
  T.tmV = c->mvV;
  T.sc = c->cg;
  T.parity = parity;
  T.zt = (const R *)c->zt;
  T.err = c->dev_err;
  T.wait = c->wait_cycles;
  const size_t smem = mv_smem_bytes<R, kMvTY, true>((int)c->mats.size());
  const dim3 blk(kMvTX, kMvTY);
  const dim3 grd((c->nx + 1 + kMvElems - 2) / (kMvElems - 1), (c->ny + 1 + kMvTY - 2) / (kMvTY - 1));
  hex8_matvec_tma_kernel<R, kMvTY, true><<<grd, blk, smem, c->stream>>>(T); ++c->launches;
  CHECK_LAUNCH(c);
  return COSIM_OK;
}

// CTAs of the TMA matvec (the one the PCG uses: its p.Kp partial sums)
static int mv_blocks(const cosim_ctx *c) {
  return ((c->nx + 1 + kMvElems - 2) / (kMvElems - 1)) * ((c->ny + 1 + kMvTY - 2) / (kMvTY - 1));
}

// Jacobi-PCG on K U = F in the context precision, U from zero, with the
// Jacobi inverse diagonal already in Dinv. Stops at ||r|| <= rtol ||F|| (the
// recursively updated residual, checked every `every` iterations) or maxit.
template <typename R>
static cosim_status pcg_run(cosim_ctx *c, double rtol, int64_t maxit, int every, int64_t *iters, double *relres,
                            bool *converged) {
  R *const *U = (R *const *)c->U;
  R *const *F = (R *const *)c->F;
  R *const *Rv = (R *const *)c->Rv;
  R *const *Pb[2] = {(R *const *)c->Pv, (R *const *)c->Pv2};  // the two direction buffers
  R *const *Pv = Pb[0];
  R *const *Qv = (R *const *)c->Qv;
  R *const *D = (R *const *)c->Dinv;
  const long long n = c->npad;
  double *pa = c->part, *pb = c->part + c->npart;
  // The iteration runs on s F, s = 2^e bringing the right-hand side's RMS
  // near one, and U is divided by s at the end: exact (a power of two), it
  // keeps small thermal loads out of the FP32 subnormal range, where the
  // residual products would underflow long before the tolerance is met.
  double scale = 1.0, bb = 0.0;
  sumsq3_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, F[0], F[1], F[2], pb); ++c->launches;
  CHECK_LAUNCH(c);
  reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pb, kRedBlocks, &c->cg->bb); ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, &c->cg->bb, 8, cudaMemcpyDeviceToHost, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  bb = c->host_scal[0];
  if (!std::isfinite(bb)) return fail(c, COSIM_ERR_NONFINITE, "non-finite right-hand side");
  if (bb > 0) scale = std::ldexp(1.0, -(int)std::lround(0.5 * std::log2(bb / (3.0 * (double)(c->nx + 1) *
                                                                                    (c->ny + 1) * (c->nz + 1)))));
  cg_init_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, F[0], F[1], F[2], D[0], D[1], D[2], U[0], U[1], U[2],
                                                       Rv[0], Rv[1], Rv[2], Pv[0], Pv[1], Pv[2], pa, pb, (R)scale);
  ++c->launches;
  CHECK_LAUNCH(c);
  reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pa, kRedBlocks, &c->cg->rz[0]); ++c->launches;
  reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pb, kRedBlocks, &c->cg->bb); ++c->launches;
  CHECK_LAUNCH(c);
  if (scale != 1.0) {  // the scaled right-hand side's norm for the relative residual
    CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, &c->cg->bb, 8, cudaMemcpyDeviceToHost, c->stream));
    CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    bb = c->host_scal[0];
    if (!std::isfinite(bb)) return fail(c, COSIM_ERR_NONFINITE, "non-finite right-hand side");
  }
  int64_t it = 0;
  *relres = bb > 0 ? 1.0 : 0.0;
  *converged = !(bb > 0);
  const int nmv = mv_blocks(c);
  // from the second iteration on, the direction update p = D^-1 r + beta p
  // runs inside the product (p alternates between the two buffers);
  // otherwise (the stages do not fit) a separate pass updates p in place
  const bool fuse = mv_dir_fits<R>(c);
  int cur = 0;  // buffer of this iteration's direction (cg_init wrote Pv)
  while (bb > 0) {
    const int parity = (int)(it & 1);
    cosim_status st;
    if (it == 0 || !fuse) {
      void *pv[3] = {Pb[cur][0], Pb[cur][1], Pb[cur][2]}, *qv[3] = {Qv[0], Qv[1], Qv[2]};
      st = matvec_t<R>(c, pv, qv, pa);
    } else {
      st = matvec_dir<R>(c, cur, parity ^ 1, pa);
      cur ^= 1;
    }
    if (st != COSIM_OK) return st;
    R *const *P = Pb[cur];
    reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pa, nmv, &c->cg->pq); ++c->launches;
    // fused: the solution's update x += alpha p waits for the next product
    // (or the final axpy), so this pass streams r, q and D only
    if (fuse)
      cg_update_kernel<R, false><<<kRedBlocks, 256, 0, c->stream>>>(n, c->cg, parity, U[0], U[1], U[2], Rv[0], Rv[1],
                                                                    Rv[2], P[0], P[1], P[2], Qv[0], Qv[1], Qv[2],
                                                                    D[0], D[1], D[2], pa, pb);
    else
      cg_update_kernel<R, true><<<kRedBlocks, 256, 0, c->stream>>>(n, c->cg, parity, U[0], U[1], U[2], Rv[0], Rv[1],
                                                                   Rv[2], P[0], P[1], P[2], Qv[0], Qv[1], Qv[2], D[0],
                                                                   D[1], D[2], pa, pb);
    ++c->launches;
    reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pa, kRedBlocks, &c->cg->rz[parity ^ 1]); ++c->launches;
    reduce_final_kernel<<<1, 1024, 0, c->stream>>>(pb, kRedBlocks, &c->cg->rr); ++c->launches;
    CHECK_LAUNCH(c);
    ++it;
    if (it % every == 0 || it >= maxit) {
      CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, &c->cg->rr, 8, cudaMemcpyDeviceToHost, c->stream));
      CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
      const double rr = c->host_scal[0];
      if (!std::isfinite(rr)) return fail(c, COSIM_ERR_NONFINITE, "non-finite CG residual");
      *relres = std::sqrt(rr / bb);
      if (*relres <= rtol) {
        *converged = true;
        break;
      }
      if (it >= maxit) break;
    }
    if (!fuse) {
      cg_direction_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->cg, parity, Pv[0], Pv[1], Pv[2], Rv[0], Rv[1],
                                                                Rv[2], D[0], D[1], D[2]); ++c->launches;
      CHECK_LAUNCH(c);
    }
  }
  *iters = it;
  const bool last_step = fuse && it > 0;
  if (last_step) {  // the last direction's step (the products applied the earlier ones), with the final scale
    cg_axpy_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->cg, (int)((it - 1) & 1), U[0], U[1], U[2], Pb[cur][0],
                                                         Pb[cur][1], Pb[cur][2], (R)(1.0 / scale));
    ++c->launches;
    CHECK_LAUNCH(c);
  }
  if (scale != 1.0 && !last_step) {
    scale3_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, U[0], U[1], U[2], (R)(1.0 / scale)); ++c->launches;
    CHECK_LAUNCH(c);
  }
  return COSIM_OK;
}

static cosim_status refine_alloc(cosim_ctx *c) {
  if (c->refine_ready) return COSIM_OK;
  for (int a = 0; a < 3; ++a) {
    ALLOC(c, c->U64[a], c->npad * 8);
    ALLOC(c, c->F64[a], c->npad * 8);
    ALLOC(c, c->R64[a], c->npad * 8);
  }
  c->refine_ready = true;
  return COSIM_OK;
}

template <typename R>
static cosim_status stress_solve_t(cosim_ctx *c, const cosim_stress_opts *o, cosim_stress_report *rep) {
  const auto t0 = std::chrono::steady_clock::now();
  const Geo<R> g = make_geo<R>(c);
  const size_t smem = c->mats.size() * M_COLS * sizeof(R);
  const dim3 blk(32, 8), grd((c->nx + 1 + 31) / 32, (c->ny + 1 + 7) / 8);  // node columns (the kernels march in z)
  R *const *U = (R *const *)c->U;
  R *const *F = (R *const *)c->F;
  R *const *D = (R *const *)c->Dinv;
  const long long n = c->npad;
  const R Tref = (R)(o->T_ref - c->T_init);  // device T is the rise over T_init
  // the temperature the load is taken from: the current field or the peak snapshot
  const R *Tsrc = (const R *)(o->temperature == COSIM_STRESS_T_PEAK ? c->T_peak : c->T[c->tpar]);
  hex8_node_kernel<R, 0><<<grd, blk, smem, c->stream>>>(g, c->mask, nullptr, Tref, D[0], D[1], D[2]); ++c->launches;
  CHECK_LAUNCH(c);
  const double rtol = o->rtol > 0 ? o->rtol : 1e-9;
  const int64_t maxit = o->maxit > 0 ? o->maxit : 200000;
  const int every = o->check_every > 0 ? o->check_every : 32;
  int64_t iters = 0, steps = 0;
  double relres = 0;
  bool converged = false;
  cosim_status result = COSIM_OK;
  if (!o->refine) {
    hex8_node_kernel<R, 1><<<grd, blk, smem, c->stream>>>(g, c->mask, Tsrc, Tref, F[0], F[1], F[2]); ++c->launches;
    CHECK_LAUNCH(c);
    cosim_status st = pcg_run<R>(c, rtol, maxit, every, &iters, &relres, &converged);
    if (st != COSIM_OK) return st;
  } else {
    // FP64 outer loop: r = f - K u with the FP64 load, FP64 matvec and FP64 u;
    // inner solves K d = r in the context precision; u += d.
    cosim_status st = refine_alloc(c);
    if (st != COSIM_OK) return st;
    const Geo<double> g64 = make_geo64(c);
    const size_t smem64 = c->mats.size() * M_COLS * sizeof(double);
    double *T64 = (double *)c->scratch;  // temperature rise in FP64
    const R *Tc = Tsrc;
    cast3_kernel<R, double><<<kRedBlocks, 256, 0, c->stream>>>(n, Tc, Tc, Tc, T64, T64, T64); ++c->launches;
    hex8_node_kernel<double, 1><<<grd, blk, smem64, c->stream>>>(g64, c->mask, T64, o->T_ref - c->T_init, c->F64[0],
                                                                 c->F64[1], c->F64[2]); ++c->launches;
    CHECK_LAUNCH(c);
    for (int a = 0; a < 3; ++a) CHECK_CUDA(c, cudaMemsetAsync(c->U64[a], 0, n * 8, c->stream));
    const double inner = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
    const int max_refine = o->max_refine > 0 ? o->max_refine : 30;
    double ff = -1;
    while (true) {
      void *u64[3] = {c->U64[0], c->U64[1], c->U64[2]}, *r64[3] = {c->R64[0], c->R64[1], c->R64[2]};
      if ((st = matvec_g<double>(c, g64, u64, r64, nullptr)) != COSIM_OK) return st;
      residual64_kernel<<<kRedBlocks, 256, 0, c->stream>>>(n, c->F64[0], c->F64[1], c->F64[2], c->R64[0], c->R64[1],
                                                            c->R64[2], c->part); ++c->launches;
      reduce_final_kernel<<<1, 1024, 0, c->stream>>>(c->part, kRedBlocks, c->scal); ++c->launches;
      CHECK_LAUNCH(c);
      CHECK_CUDA(c, cudaMemcpyAsync(c->host_scal, c->scal, 8, cudaMemcpyDeviceToHost, c->stream));
      CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
      const double rr = c->host_scal[0];
      if (!std::isfinite(rr)) return fail(c, COSIM_ERR_NONFINITE, "non-finite refinement residual");
      if (ff < 0) ff = rr;  // u = 0 on the first pass: r = f
      relres = ff > 0 ? std::sqrt(rr / ff) : 0.0;
      if (relres <= rtol) {
        converged = true;
        break;
      }
      if (steps >= max_refine) break;
      cast3_kernel<double, R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->R64[0], c->R64[1], c->R64[2], F[0], F[1],
                                                                 F[2]); ++c->launches;
      CHECK_LAUNCH(c);
      int64_t it = 0;
      double rel_in = 0;
      bool conv_in = false;
      if ((st = pcg_run<R>(c, inner, maxit, every, &it, &rel_in, &conv_in)) != COSIM_OK) return st;
      iters += it;
      ++steps;
      add_correction_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->U64[0], c->U64[1], c->U64[2], U[0], U[1],
                                                                  U[2]); ++c->launches;
      CHECK_LAUNCH(c);
    }
    cast3_kernel<double, R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->U64[0], c->U64[1], c->U64[2], U[0], U[1],
                                                               U[2]); ++c->launches;
    cast3_kernel<double, R><<<kRedBlocks, 256, 0, c->stream>>>(n, c->F64[0], c->F64[1], c->F64[2], F[0], F[1],
                                                               F[2]); ++c->launches;
    CHECK_LAUNCH(c);
  }
  if (!converged) {
    result = COSIM_ERR_NOT_CONVERGED;
    c->err = o->refine ? "refinement did not reach rtol" : "CG reached maxit";
  }
  const dim3 grc((c->nx + 31) / 32, (c->ny + 7) / 8, c->nz);
  von_mises_kernel<R><<<grc, blk, smem, c->stream>>>(g, U[0], U[1], U[2], Tsrc, Tref, (R *)c->VM); ++c->launches;
  umag_kernel<R><<<kRedBlocks, 256, 0, c->stream>>>(n, U[0], U[1], U[2], (R *)c->UMAG); ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  if (rep) {
    rep->iters = iters;
    rep->relres = relres;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->refine_steps = steps;
  }
  return result;
}

extern "C" cosim_status cosim_stress_solve(cosim_ctx *c, const cosim_stress_opts *o, cosim_stress_report *rep) {
  if (!c) return COSIM_ERR_INVALID;
  if (!o) return fail(c, COSIM_ERR_INVALID, "opts is NULL");
  if (c->nz < 1) return fail(c, COSIM_ERR_INVALID, "grid too thin");
  if (o->temperature != COSIM_STRESS_T_CURRENT && o->temperature != COSIM_STRESS_T_PEAK)
    return fail(c, COSIM_ERR_INVALID, "bad temperature source");
  if (o->temperature == COSIM_STRESS_T_PEAK && !c->T_peak)
    return fail(c, COSIM_ERR_INVALID, "no peak snapshot: run cosim_coupled_march first");
  cosim_status st = mech_alloc(c);
  if (st != COSIM_OK) return st;
  if ((st = upload_mask(c, o)) != COSIM_OK) return st;
  return c->prec == COSIM_FP64 ? stress_solve_t<double>(c, o, rep) : stress_solve_t<float>(c, o, rep);
}

extern "C" cosim_status cosim_stress_apply(cosim_ctx *c, const cosim_stress_opts *o, const void *u, void *y,
                                           int32_t on_device) {
  if (!c) return COSIM_ERR_INVALID;
  if (!o || !u || !y) return fail(c, COSIM_ERR_INVALID, "NULL argument");
  cosim_status st = mech_alloc(c);
  if (st != COSIM_OK) return st;
  if ((st = upload_mask(c, o)) != COSIM_OK) return st;
  const size_t nn = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  // stage the dense SoA input into the padded direction vector, output through Kp
  for (int a = 0; a < 3; ++a) {
    const char *src = (const char *)u + a * nn * c->rsz;
    CHECK_CUDA(c, cudaMemcpy2DAsync(c->Pv[a], c->px * c->rsz, src, (c->nx + 1) * c->rsz, (c->nx + 1) * c->rsz,
                                    (size_t)(c->ny + 1) * (c->nz + 1),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  st = c->prec == COSIM_FP64 ? matvec_t<double>(c, c->Pv, c->Qv, nullptr) : matvec_t<float>(c, c->Pv, c->Qv, nullptr);
  if (st != COSIM_OK) return st;
  for (int a = 0; a < 3; ++a) {
    char *dst = (char *)y + a * nn * c->rsz;
    CHECK_CUDA(c, cudaMemcpy2DAsync(dst, (c->nx + 1) * c->rsz, c->Qv[a], c->px * c->rsz, (c->nx + 1) * c->rsz,
                                    (size_t)(c->ny + 1) * (c->nz + 1),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return COSIM_OK;
}

// ---------------------------------------------------------------- field I/O

// dense <-> padded copies with type conversion. For E/H fields on write,
// entries that are not unknowns are stored as zero. A block walks whole rows
// (no per-element index division); a temperature offset is added in the
// output precision when both sides are FP32 (the FP64 addition per element
// it replaces is slow on this part; the sum of two FP32 values rounds once).
template <typename S, typename D>
__global__ void pack_kernel(const S *src, D *dst, int nx1, int ny1, int nz1, int px, double add) {
  const long long rows = (long long)ny1 * nz1;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const S *s = src + r * px;
    D *d = dst + r * nx1;
    for (int i = threadIdx.x; i < nx1; i += blockDim.x) {
      if (add == 0.0)
        d[i] = (D)s[i];
      else if constexpr (sizeof(S) == 4 && sizeof(D) == 4)
        d[i] = s[i] + (float)add;
      else
        d[i] = (D)((double)s[i] + add);
    }
  }
}

struct FieldMask {  // which node-sized entries of an E/H field are unknowns
  int kind;         // -1 none, 0..2 E axis, 3..5 H axis
  int n[3];
  int fixlo[3], fixhi[3];
  __device__ bool keep(int i, int j, int k) const {
    if (kind < 0) return true;
    const int p[3] = {i, j, k};
    const int a = kind % 3;
    if (kind < 3) {
      if (p[a] >= n[a]) return false;
      for (int b = 0; b < 3; ++b) {
        if (b == a) continue;
        if ((p[b] == 0 && fixlo[b]) || (p[b] == n[b] && fixhi[b])) return false;
      }
      return true;
    }
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    return p[b] < n[b] && p[cc] < n[cc];
  }
};

template <typename S, typename D>
__global__ void unpack_kernel(const S *src, D *dst, int nx1, int ny1, int nz1, int px, FieldMask fm, double sub) {
  const long long rows = (long long)ny1 * nz1;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {  // a block walks whole rows
    const int j = (int)(r % ny1), k = (int)(r / ny1);
    const S *s = src + r * nx1;
    D *d = dst + r * px;
    for (int i = threadIdx.x; i < nx1; i += blockDim.x)
      d[i] = fm.keep(i, j, k) ? (sub != 0.0 ? (D)((double)s[i] - sub) : (D)s[i]) : D(0);
  }
}

static void *field_ptr(cosim_ctx *c, int f, int *elem_bytes, bool *cells, bool *is_double) {
  *cells = false;
  *is_double = c->prec == COSIM_FP64;
  *elem_bytes = (int)c->rsz;
  switch (f) {
    case COSIM_F_EX: case COSIM_F_EY: case COSIM_F_EZ: return c->E[c->par][f];
    case COSIM_F_HX: case COSIM_F_HY: case COSIM_F_HZ: return c->H[c->par][f - 3];
    case COSIM_F_T: case COSIM_F_DT: return c->T[c->tpar];
    case COSIM_F_T_PEAK: return c->T_peak;
    case COSIM_F_Q: *is_double = true; *elem_bytes = 8; return c->Q;
    case COSIM_F_P: return c->P;
    case COSIM_F_UX: case COSIM_F_UY: case COSIM_F_UZ: return c->mech_ready ? c->U[f - COSIM_F_UX] : nullptr;
    case COSIM_F_VM: *cells = true; return c->mech_ready ? c->VM : nullptr;
    case COSIM_F_UMAG: return c->mech_ready ? c->UMAG : nullptr;
    case COSIM_F_FX: case COSIM_F_FY: case COSIM_F_FZ: return c->mech_ready ? c->F[f - COSIM_F_FX] : nullptr;
    default: return nullptr;
  }
}

template <typename S, typename D>
static void launch_pack(cosim_ctx *c, const void *src, void *dst, bool cells, double add) {
  const int nx1 = cells ? c->nx : c->nx + 1, ny1 = cells ? c->ny : c->ny + 1, nz1 = cells ? c->nz : c->nz + 1;
  const int px = cells ? c->nx : c->px;
  pack_kernel<S, D><<<kRedBlocks, 256, 0, c->stream>>>((const S *)src, (D *)dst, nx1, ny1, nz1, px, add); ++c->launches;
}

// the dense copy of a field in dtype at out (device), on the context's stream
static cosim_status pack_field(cosim_ctx *c, int32_t field, int32_t dtype, void *out) {
  int eb;
  bool cells, sdbl;
  void *src = field_ptr(c, field, &eb, &cells, &sdbl);
  if (field == COSIM_F_Q) {
    cosim_status fs = joule_flush(c);
    if (fs != COSIM_OK) return fs;
  }
  const double add = (field == COSIM_F_T || field == COSIM_F_T_PEAK) ? c->T_init : 0.0;
  if (sdbl && dtype == COSIM_FP64) launch_pack<double, double>(c, src, out, cells, add);
  else if (sdbl) launch_pack<double, float>(c, src, out, cells, add);
  else if (dtype == COSIM_FP64) launch_pack<float, double>(c, src, out, cells, add);
  else launch_pack<float, float>(c, src, out, cells, add);
  CHECK_LAUNCH(c);
  return COSIM_OK;
}

// argument checks shared by the read calls: the field exists and dst has its size
static cosim_status check_read(cosim_ctx *c, int32_t field, int32_t dtype, const void *dst, size_t bytes) {
  int eb;
  bool cells, sdbl;
  if (!field_ptr(c, field, &eb, &cells, &sdbl)) return fail(c, COSIM_ERR_INVALID, "unknown field, or field not computed yet");
  if (dtype != COSIM_FP64 && dtype != COSIM_FP32) return fail(c, COSIM_ERR_INVALID, "bad dtype");
  const size_t n = cells ? (size_t)c->nx * c->ny * c->nz : (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  const size_t ob = dtype == COSIM_FP64 ? 8 : 4;
  if (!dst || bytes != n * ob) return fail(c, COSIM_ERR_INVALID, "dst size mismatch");
  return COSIM_OK;
}

// A kernel whose bounded wait for staged data expired sets c->dev_err; report it
// (and clear it) at the next synchronising call.
static cosim_status check_device_wait(cosim_ctx *c) {
  int h = 0;
  CHECK_CUDA(c, cudaMemcpy(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h == 0) return COSIM_OK;
  CHECK_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
  return fail(c, COSIM_ERR_TIMEOUT, h == 2 ? "EM kernel: a TMA alignment precondition failed; no step was taken"
                                           : "a bounded in-kernel wait for staged data expired; results are invalid");
}

extern "C" cosim_status cosim_read_fields(cosim_ctx *c, int32_t field, int32_t dtype, void *dst, size_t bytes,
                                          int32_t dst_is_device) {
  if (!c) return COSIM_ERR_INVALID;
  cosim_status st = check_read(c, field, dtype, dst, bytes);
  if (st != COSIM_OK) return st;
  void *out = dst_is_device ? dst : c->scratch;
  if ((st = pack_field(c, field, dtype, out)) != COSIM_OK) return st;
  if (!dst_is_device) CHECK_CUDA(c, cudaMemcpyAsync(dst, c->scratch, bytes, cudaMemcpyDeviceToHost, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_wait(c);
}

extern "C" cosim_status cosim_read_fields_async(cosim_ctx *c, int32_t field, int32_t dtype, void *dst, size_t bytes,
                                                int32_t dst_is_device) {
  if (!c) return COSIM_ERR_INVALID;
  cosim_status st = check_read(c, field, dtype, dst, bytes);
  if (st != COSIM_OK) return st;
  if (!c->rd_stream) {
    CHECK_CUDA(c, cudaStreamCreateWithFlags(&c->rd_stream, cudaStreamNonBlocking));
    CHECK_CUDA(c, cudaEventCreateWithFlags(&c->rd_packed, cudaEventDisableTiming));
    CHECK_CUDA(c, cudaEventCreateWithFlags(&c->rd_done, cudaEventDisableTiming));
  }
  if (c->rd_bytes < bytes) {  // the largest read so far: node-sized FP64 at most
    const size_t cap = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1) * 8;
    if (c->rd_pending) CHECK_CUDA(c, cudaEventSynchronize(c->rd_done));
    ALLOC(c, c->rd_stage, cap);
    c->rd_bytes = cap;
  }
  // the staging buffer is free once the previous copy has landed
  if (c->rd_pending) CHECK_CUDA(c, cudaStreamWaitEvent(c->stream, c->rd_done, 0));
  if ((st = pack_field(c, field, dtype, c->rd_stage)) != COSIM_OK) return st;
  CHECK_CUDA(c, cudaEventRecord(c->rd_packed, c->stream));
  CHECK_CUDA(c, cudaStreamWaitEvent(c->rd_stream, c->rd_packed, 0));
  CHECK_CUDA(c, cudaMemcpyAsync(dst, c->rd_stage, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->rd_stream));
  CHECK_CUDA(c, cudaEventRecord(c->rd_done, c->rd_stream));
  c->rd_pending = true;
  return COSIM_OK;
}

extern "C" cosim_status cosim_wait_reads(cosim_ctx *c) {
  if (!c) return COSIM_ERR_INVALID;
  if (!c->rd_pending) return COSIM_OK;
  CHECK_CUDA(c, cudaEventSynchronize(c->rd_done));
  c->rd_pending = false;
  return check_device_wait(c);
}

extern "C" cosim_status cosim_write_fields(cosim_ctx *c, int32_t field, int32_t dtype, const void *src, size_t bytes,
                                           int32_t src_is_device) {
  if (!c) return COSIM_ERR_INVALID;
  if (field == COSIM_F_VM || field == COSIM_F_UMAG || (field >= COSIM_F_FX && field <= COSIM_F_FZ) ||
      field == COSIM_F_T_PEAK)
    return fail(c, COSIM_ERR_INVALID, "field is not writable");
  if (field >= COSIM_F_UX && field <= COSIM_F_UZ) {
    cosim_status st = mech_alloc(c);
    if (st != COSIM_OK) return st;
  }
  int eb;
  bool cells, ddbl;
  void *dst = field_ptr(c, field, &eb, &cells, &ddbl);
  if (!dst) return fail(c, COSIM_ERR_INVALID, "unknown field");
  if (dtype != COSIM_FP64 && dtype != COSIM_FP32) return fail(c, COSIM_ERR_INVALID, "bad dtype");
  const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  const size_t ib = dtype == COSIM_FP64 ? 8 : 4;
  if (!src || bytes != n * ib) return fail(c, COSIM_ERR_INVALID, "src size mismatch");
  if (field == COSIM_F_Q) {  // the written values replace the whole accumulated energy
    CHECK_CUDA(c, cudaMemsetAsync(c->Qs, 0, c->npad * c->rsz, c->stream));
    c->qs_dirty = false;
  }
  const void *in = src;
  if (!src_is_device) {
    CHECK_CUDA(c, cudaMemcpyAsync(c->scratch, src, bytes, cudaMemcpyHostToDevice, c->stream));
    in = c->scratch;
  }
  FieldMask fm;
  fm.kind = field <= COSIM_F_HZ ? field : -1;
  for (int a = 0; a < 3; ++a) {
    fm.n[a] = n_of(c, a);
    fm.fixlo[a] = c->em_bc[2 * a] != COSIM_BC_PMC;
    fm.fixhi[a] = c->em_bc[2 * a + 1] != COSIM_BC_PMC;
  }
  const int nx1 = c->nx + 1, ny1 = c->ny + 1, nz1 = c->nz + 1;
  const double sub = field == COSIM_F_T ? c->T_init : 0.0;
  if (ddbl && dtype == COSIM_FP64)
    unpack_kernel<double, double><<<kRedBlocks, 256, 0, c->stream>>>((const double *)in, (double *)dst, nx1, ny1, nz1, c->px, fm, sub);
  else if (ddbl)
    unpack_kernel<float, double><<<kRedBlocks, 256, 0, c->stream>>>((const float *)in, (double *)dst, nx1, ny1, nz1, c->px, fm, sub);
  else if (dtype == COSIM_FP64)
    unpack_kernel<double, float><<<kRedBlocks, 256, 0, c->stream>>>((const double *)in, (float *)dst, nx1, ny1, nz1, c->px, fm, sub);
  else
    unpack_kernel<float, float><<<kRedBlocks, 256, 0, c->stream>>>((const float *)in, (float *)dst, nx1, ny1, nz1, c->px, fm, sub);
  ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return COSIM_OK;
}

// ---------------------------------------------------------------- autotuning

// tuned (EM tile height, thermal block height) per (nx, ny, nz, precision)
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;

template <typename R>
static cosim_status autotune_t(cosim_ctx *c, int *em_ty, int *th_by) {
  cudaEvent_t e0, e1;
  CHECK_CUDA(c, cudaEventCreate(&e0));
  CHECK_CUDA(c, cudaEventCreate(&e1));
  cosim_status st = COSIM_OK;
  auto time_ms = [&](auto &&launch, int reps) -> float {
    float ms = 1e30f;
    if ((st = launch(2)) != COSIM_OK) return ms;  // warm-up
    cudaEventRecord(e0, c->stream);
    if ((st = launch(reps)) != COSIM_OK) return ms;
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  // EM tile height (FP32 plain steps): probe launches leave the state as it is
  int best_ty = kEmTY;
  if constexpr (sizeof(R) == 4) {
    const float t8 = time_ms([&](int n) { return em_steps_tile<R, kEmTY>(c, n, false, false, false, true); }, 5);
    const float t4 = time_ms([&](int n) { return em_steps_tile<R, kEmTYSmall>(c, n, false, false, false, true); }, 5);
    if (st == COSIM_OK && t4 < t8) best_ty = kEmTYSmall;
  }
  // thermal step kernel (TMA tiles, or the classic kernel with 4/8/16-row
  // blocks): dt = 0 launches write the spare buffer with T itself
  const int keep_by = c->th_by;
  int best_by = 0;
  float best = 1e30f;
  for (int by : {0, 4, 8, 16}) {
    c->th_by = by;
    const float t = time_ms(
        [&](int n) {
          for (int q = 0; q < n; ++q) {
            const cosim_status ts = launch_thermal<R>(c, R(0), false);
            if (ts != COSIM_OK) return ts;
          }
          return COSIM_OK;
        },
        5);
    if (t < best) best = t, best_by = by;
  }
  c->th_by = keep_by;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != COSIM_OK) return st;
  *em_ty = best_ty;
  *th_by = best_by;
  return COSIM_OK;
}

extern "C" cosim_status cosim_autotune(cosim_ctx *c, uint32_t flags, int32_t *em_tile_y, int32_t *th_block_y) {
  if (!c) return COSIM_ERR_INVALID;
  if (flags & ~(COSIM_TUNE_FORCE | COSIM_TUNE_FIXED)) return fail(c, COSIM_ERR_INVALID, "bad autotune flags");
  const auto key = std::make_tuple(c->nx, c->ny, c->nz, (int)c->prec);
  int ty = 0, by = 0;
  if (flags & COSIM_TUNE_FIXED) {
    if (!em_tile_y || !th_block_y) return fail(c, COSIM_ERR_INVALID, "FIXED needs both heights");
    ty = *em_tile_y, by = *th_block_y;
    const bool ok_ty = ty == kEmTY || (ty == kEmTYSmall && c->prec != COSIM_FP64);
    if (!ok_ty || (by != 0 && by != 4 && by != 8 && by != 16))
      return fail(c, COSIM_ERR_INVALID, "unsupported launch shape");
    CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graph(c);
    c->em_ty = ty;
    c->th_by = by;
    return COSIM_OK;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end() && !(flags & COSIM_TUNE_FORCE)) ty = it->second.first, by = it->second.second;
  }
  if (ty == 0) {
    CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    const cosim_status st = c->prec == COSIM_FP64 ? autotune_t<double>(c, &ty, &by) : autotune_t<float>(c, &ty, &by);
    if (st != COSIM_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {ty, by};
  }
  drop_graph(c);  // a captured graph holds the old launch shapes
  c->em_ty = ty;
  c->th_by = by;
  if (em_tile_y) *em_tile_y = ty;
  if (th_block_y) *th_block_y = by;
  return COSIM_OK;
}

// ---------------------------------------------------------------- options, health check, checkpoints

extern "C" cosim_status cosim_set_option(cosim_ctx *c, int32_t what, double value) {
  if (!c) return COSIM_ERR_INVALID;
  if (what == COSIM_OPT_WAIT_CYCLES) {
    if (!(value >= 1000.0 && value <= 9.0e18)) return fail(c, COSIM_ERR_INVALID, "wait bound out of range");
    c->wait_cycles = (long long)value;
    drop_graph(c);  // a captured graph holds the old bound
    return COSIM_OK;
  }
  return fail(c, COSIM_ERR_INVALID, "unknown option");
}

// One CTA waits for a barrier phase that needs two arrivals and gets one:
// the bounded wait runs out after `limit` cycles and takes the solver
// kernels' error path (the context's error word).
__global__ void wait_selftest_kernel(int *err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    fence_mbar_init();
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
    if (!mbar_wait(&bar, 0u, limit)) atomicExch(err, 1);
  }
}

extern "C" cosim_status cosim_wait_selftest(cosim_ctx *c) {
  if (!c) return COSIM_ERR_INVALID;
  cosim_status st = check_device_wait(c);  // an earlier expiry is reported first
  if (st != COSIM_OK) return st;
  wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->dev_err, c->wait_cycles); ++c->launches;
  CHECK_LAUNCH(c);
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_wait(c);
}

// Checkpoint layout: this header, then the arrays in a fixed order (E and H
// of the current parity, the CPML auxiliaries present, the short Joule
// window, the FP64 Joule total, the temperature, the thermal source).
struct CkHeader {
  char magic[8];
  int32_t version, prec, nx, ny, nz, px, L, par, tpar, qs_dirty;
  int64_t npad, psi_len[3], step, n_acc, dstep;
};

static std::vector<std::pair<void *, size_t>> ck_arrays(cosim_ctx *c, int par, int tpar) {
  std::vector<std::pair<void *, size_t>> v;
  const size_t nb = (size_t)c->npad * c->rsz;
  for (int a = 0; a < 3; ++a) v.emplace_back(c->E[par][a], nb);
  for (int a = 0; a < 3; ++a) v.emplace_back(c->H[par][a], nb);
  for (int a = 0; a < 3; ++a)
    for (int s2 = 0; s2 < 2; ++s2)
      if (c->psi_len[a] > 0) {  // x / y: records; z: separate arrays
        const size_t pb = (size_t)c->psi_len[a] * (a < 2 ? 16 : c->rsz);
        for (void *q : {c->xE[par][a][s2], c->dE[par][a][s2], c->xH[par][a][s2], c->dH[par][a][s2],
                        c->lE[par][a][s2], c->lH[par][a][s2]})
          if (q) v.emplace_back(q, pb);
      }
  v.emplace_back(c->Qs, nb);
  v.emplace_back(c->Q, (size_t)c->npad * 8);
  v.emplace_back(c->T[tpar], nb);
  v.emplace_back(c->P, nb);
  return v;
}

extern "C" cosim_status cosim_checkpoint_size(const cosim_ctx *c, size_t *bytes) {
  if (!c || !bytes) return COSIM_ERR_INVALID;
  size_t n = sizeof(CkHeader);
  for (auto &a : ck_arrays(const_cast<cosim_ctx *>(c), c->par, c->tpar)) n += a.second;
  *bytes = n;
  return COSIM_OK;
}

extern "C" cosim_status cosim_checkpoint_save(cosim_ctx *c, void *dst, size_t bytes, int32_t dst_is_device) {
  if (!c) return COSIM_ERR_INVALID;
  size_t need = 0;
  cosim_checkpoint_size(c, &need);
  if (!dst || bytes != need) return fail(c, COSIM_ERR_INVALID, "checkpoint buffer size mismatch");
  CkHeader h{};
  std::memcpy(h.magic, "COSIMCK1", 8);
  h.version = 2, h.prec = c->prec, h.nx = c->nx, h.ny = c->ny, h.nz = c->nz, h.px = c->px, h.L = c->L;
  h.par = c->par, h.tpar = c->tpar, h.qs_dirty = c->qs_dirty ? 1 : 0;
  h.npad = c->npad, h.step = c->step, h.n_acc = c->n_acc;
  for (int a = 0; a < 3; ++a) h.psi_len[a] = c->psi_len[a];
  const cudaMemcpyKind kd = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  long long dstep = 0;
  CHECK_CUDA(c, cudaMemcpyAsync(&dstep, c->dstep, 8, cudaMemcpyDeviceToHost, c->stream));
  char *o = (char *)dst + sizeof(CkHeader);
  for (auto &a : ck_arrays(c, c->par, c->tpar)) {
    CHECK_CUDA(c, cudaMemcpyAsync(o, a.first, a.second, kd, c->stream));
    o += a.second;
  }
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  h.dstep = dstep;
  CHECK_CUDA(c, cudaMemcpy(dst, &h, sizeof h, dst_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
  return check_device_wait(c);
}

extern "C" cosim_status cosim_checkpoint_load(cosim_ctx *c, const void *src, size_t bytes, int32_t src_is_device) {
  if (!c) return COSIM_ERR_INVALID;
  if (!src || bytes < sizeof(CkHeader)) return fail(c, COSIM_ERR_INVALID, "checkpoint too short");
  CkHeader h{};
  CHECK_CUDA(c, cudaMemcpy(&h, src, sizeof h, src_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  bool same = std::memcmp(h.magic, "COSIMCK1", 8) == 0 && h.version == 2 && h.prec == c->prec && h.nx == c->nx &&
              h.ny == c->ny && h.nz == c->nz && h.px == c->px && h.L == c->L && h.npad == c->npad &&
              (h.par == 0 || h.par == 1) && (h.tpar == 0 || h.tpar == 1);
  for (int a = 0; a < 3; ++a) same = same && h.psi_len[a] == c->psi_len[a];
  if (!same) return fail(c, COSIM_ERR_INVALID, "checkpoint of another grid, precision or CPML set-up");
  size_t need = sizeof(CkHeader);
  for (auto &a : ck_arrays(c, h.par, h.tpar)) need += a.second;
  if (bytes != need) return fail(c, COSIM_ERR_INVALID, "checkpoint size mismatch");
  drop_graph(c);
  const cudaMemcpyKind kd = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const char *p = (const char *)src + sizeof(CkHeader);
  for (auto &a : ck_arrays(c, h.par, h.tpar)) {
    CHECK_CUDA(c, cudaMemcpyAsync(a.first, p, a.second, kd, c->stream));
    p += a.second;
  }
  const long long dstep = h.dstep;
  CHECK_CUDA(c, cudaMemcpyAsync(c->dstep, &dstep, 8, cudaMemcpyHostToDevice, c->stream));
  CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
  c->par = h.par, c->tpar = h.tpar, c->qs_dirty = h.qs_dirty != 0, c->step = h.step, c->n_acc = h.n_acc;
  return COSIM_OK;
}

extern "C" cosim_status cosim_query(const cosim_ctx *c, int32_t what, double *out) {
  if (!c || !out) return COSIM_ERR_INVALID;
  switch (what) {
    case COSIM_Q_DT_EM: *out = c->dt; break;
    case COSIM_Q_DT_TH_LIMIT: {
      cosim_status st = ensure_th_limit(const_cast<cosim_ctx *>(c));
      if (st != COSIM_OK) return st;
      *out = c->dt_th_limit;
      break;
    }
    case COSIM_Q_STEP: *out = (double)c->step; break;
    case COSIM_Q_BYTES_RESIDENT: *out = (double)c->bytes; break;
    case COSIM_Q_JOULE_STEPS: *out = (double)c->n_acc; break;
    case COSIM_Q_N_CELLS: *out = (double)c->nx * c->ny * c->nz; break;
    case COSIM_Q_N_NODES: *out = (double)(c->nx + 1) * (c->ny + 1) * (c->nz + 1); break;
    case COSIM_Q_PRECISION: *out = c->prec; break;
    case COSIM_Q_LAUNCHES: *out = (double)c->launches; break;
    case COSIM_Q_EM_TILE_Y: *out = c->prec == COSIM_FP64 ? kEmTY : c->em_ty; break;
    case COSIM_Q_TH_BLOCK_Y: *out = c->th_by; break;
    default: return COSIM_ERR_INVALID;
  }
  return COSIM_OK;
}

// ---------------------------------------------------------------- allocation-free sum
//
// For callers that cannot allocate device memory themselves: an application
// whose device memory is fully reserved by its own pool or budget, or a
// latency-critical loop in which the implicit synchronisation and possible
// failure of cudaMalloc/cudaFree are not acceptable. The two-stage reduction
// below is the same kernel pair that cosim_joule_accumulate uses for its total,
// but its partial sums live in a fixed array in this library's device image
// instead of in context-owned scratch.
namespace {
constexpr int kNoAllocMaxBlocks = 65536;                 // partial sums held by the array
constexpr long long kNoAllocPerBlock = 256LL * 16;       // elements reduced by one CTA
constexpr long long kNoAllocMaxN = kNoAllocMaxBlocks * kNoAllocPerBlock;  // 2^28 elements
// 65,536 partials + 32 doubles (the result sits at index kNoAllocMaxBlocks): 512.25 KiB,
// resident on every device that loads the library until the process exits
__device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 32];
std::mutex g_noalloc_mu;
std::vector<double *> g_noalloc_addr;  // per device: device address of g_noalloc_scratch
}  // namespace

extern "C" cosim_status cosim_sum_f64_noalloc(const double *x, int64_t n, double *out, int32_t out_is_device,
                                              void *stream) {
  g_create_error.clear();
  if (!x || !out || n < 0) {
    g_create_error = "cosim_sum_f64_noalloc: NULL pointer or negative n";
    return COSIM_ERR_INVALID;
  }
  if (n > kNoAllocMaxN) {
    g_create_error = "cosim_sum_f64_noalloc: n = " + std::to_string((long long)n) +
                     " exceeds the allocation-free limit of " + std::to_string(kNoAllocMaxN) + " elements";
    return COSIM_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return COSIM_ERR_CUDA;
  }
  double *scratch = nullptr;
  {
    // set-up once per device, with that device current: resolve the array's
    // device address (a host-side use of the symbol itself is not a device address)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= dev) g_noalloc_addr.resize(dev + 1, nullptr);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_create_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return COSIM_ERR_CUDA;
      }
      g_noalloc_addr[dev] = (double *)p;
    }
    scratch = g_noalloc_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (int)std::max<long long>(1, (n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
  // every partial slot in [0, nblk) and the result slot are written before they
  // are read, so the array needs no clearing between calls
  sum_partial_kernel<<<nblk, 256, 0, s>>>(n, x, scratch);
  reduce_final_kernel<<<1, 1024, 0, s>>>(scratch, nblk, scratch + kNoAllocMaxBlocks);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + kNoAllocMaxBlocks, sizeof(double),
                        out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !out_is_device) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_create_error = std::string("cosim_sum_f64_noalloc: ") + cudaGetErrorString(e);
    return COSIM_ERR_CUDA;
  }
  return COSIM_OK;
}
