// Device-side definitions shared by the solver kernels.
//
// Data layout in HBM (one context):
//   * node-sized fields (E, H, T, Q, P, displacement, CG vectors): dense
//     3-D arrays, x fastest, row pitch `px` = nx+1 rounded up to 32 elements
//     (128-byte aligned rows for FP32), planes of px*(ny+1) elements; the
//     padding columns i > nx are kept at zero;
//   * voxel materials: uint8, x fastest, row pitch vpx = nx rounded up to 16
//     bytes (TMA needs 16-byte strides), planes of vpx*ny (1 byte per cell);
//   * per-axis spacing tables h, 1/h, 1/dual-length (a few KB);
//   * a per-material constant table staged in shared memory by each kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cosim {

constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
constexpr int kMaxMat = 256;
constexpr int kMaxL = 32;                 // largest CPML thickness in cells
constexpr int kMaxSlab = 2 * (kMaxL + 1); // positions of both CPML slabs on one axis

// columns of the device material table (derived once per context)
enum : int {
  M_EPS = 0,   // eps0 * eps_r
  M_SDT2 = 1,  // sigma * dt_em / 2
  M_IMU = 2,   // 1 / (mu0 mu_r)
  M_K = 3,     // thermal conductivity
  M_RHOCP = 4, // volumetric heat capacity
  M_LAM = 5,   // Lame lambda
  M_MU = 6,    // Lame mu (shear modulus)
  M_BETA = 7,  // (3 lambda + 2 mu) alpha_L: thermal stress per kelvin
  M_TCR = 8,   // alpha: temperature coefficient of resistance
  M_TC0 = 9,   // 1 + alpha (T_init - T0): sigma(T) = sigma0 / (M_TC0 + M_TCR (T - T_init))
  M_COLS = 12  // (two spare columns keep rows 16-byte aligned)
};

template <typename R>
struct Geo {
  int nx, ny, nz;
  int px;              // x pitch of node arrays
  long long plane;     // px * (ny + 1)
  const uint8_t *mat;  // nz planes of ny rows of pitch vpx
  int vpx;             // voxel row pitch (bytes)
  const R *h[3];       // cell sizes, n entries per axis
  const R *ih[3];      // 1 / cell size, n entries
  const R *idual[3];   // 1 / dual length at nodes, n + 1 entries
  const R *mtab;       // nmat * M_COLS
  int nmat;

  __device__ __forceinline__ long long nid(int i, int j, int k) const {
    return (long long)k * plane + (long long)j * px + i;
  }
  // material of voxel (i,j,k), or -1 outside the grid
  __device__ __forceinline__ int cell(int i, int j, int k) const {
    return (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz)
               ? (int)__ldg(mat + ((long long)k * ny + j) * vpx + i)
               : -1;
  }
};

// material constant with a zero for "no voxel"
template <typename R>
__device__ __forceinline__ R mconst(const R *s_mt, int m, int col) {
  return m >= 0 ? s_mt[m * M_COLS + col] : R(0);
}

// stage the material table into shared memory (call by all threads, then sync)
template <typename R>
__device__ __forceinline__ void stage_table(R *dst, const R *src, int n) {
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  for (int q = t; q < n; q += nt) dst[q] = src[q];
}

// Asynchronous global -> shared copy of N (4 or 8) bytes; when ok is false the
// destination is zero-filled and nothing is read (src must still be a valid
// address). Completion is tracked with commit/wait groups.
template <int N>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, bool ok) {
  static_assert(N == 4 || N == 8 || N == 16, "cp.async size");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = ok ? N : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(N), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// a compile-time flag passed to a generic lambda
template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

// ---- Tensor-memory-accelerator (TMA) copies tracked by a shared-memory
// mbarrier (PTX ISA: cp.async.bulk.tensor, mbarrier). The CTA is its own
// cluster, so its shared::cta addresses are valid shared::cluster addresses.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}
// end the life of an initialised barrier (before its memory is initialised again)
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// order this thread's earlier shared-memory accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// one arrival that also announces `bytes` of transactions for the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// box of a 3-D tensor map at element coordinates (x, y, z) -> dst; x * element
// size must be a multiple of 16 bytes (coordinates may be negative or past the
// end: those elements are filled with zero)
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// 1-D box of a rank-1 tensor map at element x (same alignment rule as above)
__device__ __forceinline__ void tma_load_1d(void *dst, const void *tmap, int x, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(smem_u32(bar))
      : "memory");
}
// contiguous bulk copy (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// A TMA destination in shared memory must be 128-byte aligned: every staged
// box is padded to a multiple of 128 bytes.
template <typename R, int ROWS, int BX>
struct alignas(128) EmBox {
  R v[ROWS][BX];
};

// Wait for the phase of parity `parity` to complete; gives up (returns false)
// after `limit` SM clock cycles (by default about a second) so that a lost
// copy cannot hang the GPU.
constexpr long long kWaitCycles = 2LL << 30;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// ---- Arithmetic written once for one node (R) or two adjacent nodes (the
// pair type R2: float2 / double2). Every operation rounds once, to nearest,
// and the pair forms act element by element (FP32 pairs use the packed FP32
// instructions of sm_100 and later, one instruction for both nodes; FP64
// pairs are two scalar operations). The scalar forms are never contracted;
// the code generator does contract a packed product that feeds a packed
// addition into one FMA, so a formula with such a step can round a pair one
// FP32 rounding apart from the single-node form. Formulas that feed no
// product into an addition (the thermal step) give the same bits either way.
template <typename R>
struct Pair2;
template <>
struct Pair2<float> {
  using T = float2;
};
template <>
struct Pair2<double> {
  using T = double2;
};
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
// a - b, evaluated as a + (-b) (the same IEEE result)
__device__ __forceinline__ float sub_(float a, float b) { return __fadd_rn(a, -b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dadd_rn(a, -b); }
__device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ double2 fma_(double2 a, double2 b, double2 c) {
  return make_double2(fma_(a.x, b.x, c.x), fma_(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 mul_(double2 a, double2 b) { return make_double2(mul_(a.x, b.x), mul_(a.y, b.y)); }
__device__ __forceinline__ double2 add_(double2 a, double2 b) { return make_double2(add_(a.x, b.x), add_(a.y, b.y)); }
__device__ __forceinline__ double2 sub_(double2 a, double2 b) { return make_double2(sub_(a.x, b.x), sub_(a.y, b.y)); }
__device__ __forceinline__ float neg_(float a) { return -a; }
__device__ __forceinline__ double neg_(double a) { return -a; }
__device__ __forceinline__ float2 neg_(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 neg_(double2 a) { return make_double2(-a.x, -a.y); }
// load / store of V at p (a pair: two adjacent elements, p aligned to the pair)
template <typename V, typename R>
__device__ __forceinline__ V ldv_(const R *p) {
  return *reinterpret_cast<const V *>(p);
}
template <typename V, typename R>
__device__ __forceinline__ void stv_(R *p, const V &v) {
  *reinterpret_cast<V *>(p) = v;
}
// broadcast a scalar to V (a scalar or a pair)
__device__ __forceinline__ void splat_(float s, float &v) { v = s; }
__device__ __forceinline__ void splat_(float s, float2 &v) { v = make_float2(s, s); }
__device__ __forceinline__ void splat_(double s, double &v) { v = s; }
__device__ __forceinline__ void splat_(double s, double2 &v) { v = make_double2(s, s); }
template <typename V, typename R>
__device__ __forceinline__ V bc_(R s) {
  V v;
  splat_(s, v);
  return v;
}
// Reciprocal of a positive normal number: in FP32 the hardware approximation
// refined by one Newton-Raphson step, r' = r + r (1 - x r) (within about an
// ulp of 1/x); in FP64 the correctly rounded quotient.
__device__ __forceinline__ float rcp_approx_(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_(float x) {
  const float r = rcp_approx_(x);
  return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float2 rcp_(float2 x) {
  const float2 r = make_float2(rcp_approx_(x.x), rcp_approx_(x.y));
  return __ffma2_rn(r, __ffma2_rn(make_float2(-x.x, -x.y), r, make_float2(1.0f, 1.0f)), r);
}
__device__ __forceinline__ double2 rcp_(double2 x) { return make_double2(rcp_(x.x), rcp_(x.y)); }

// Sum of v over the block (any shape up to 1024 threads); the result is valid
// in thread 0. Fixed summation order: deterministic run to run.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_warp[32];
  const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // s_warp may still be read by a previous call
  if ((t & 31) == 0) s_warp[t >> 5] = v;
  __syncthreads();
  if (t < 32) {
    v = (t < (nt + 31) / 32) ? s_warp[t] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

}  // namespace cosim
