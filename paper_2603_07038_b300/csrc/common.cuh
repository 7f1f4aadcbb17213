// Device-side definitions shared by the solver kernels.
//
// Data layout in HBM (one context):
//   * node-sized fields (E, H, T, Q, P, displacement, CG vectors): dense
//     3-D arrays, x fastest, row pitch `px` = nx+1 rounded up to 32 elements
//     (128-byte aligned rows for FP32), planes of px*(ny+1) elements; the
//     padding columns i > nx are kept at zero;
//   * voxel materials: uint8 nz*ny*nx, x fastest (1 byte per cell);
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
  M_COLS = 8
};

template <typename R>
struct Geo {
  int nx, ny, nz;
  int px;              // x pitch of node arrays
  long long plane;     // px * (ny + 1)
  const uint8_t *mat;  // nz * ny * nx
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
               ? (int)__ldg(mat + ((long long)k * ny + j) * nx + i)
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
  static_assert(N == 4 || N == 8, "cp.async size");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = ok ? N : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(N), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

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
