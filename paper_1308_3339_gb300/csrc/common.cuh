// Internal declarations of the fmmpc CUDA library (not part of the ABI).
//
// Geometry is kept in node units: node (i, j), 0-based, sits at (i+1, j+1); a cell at
// level l has width rho_l = n >> l nodes.  Expansions are stored scaled,
// Mt_k = M_k / rho^k and Lt_k = L_k rho^k, so every translation works on O(1) numbers.
// The physical kernel is G = -(1/2pi)(ln h + ln|d|_node); the ln h part is a constant
// times the total source weight and is added once, through the root local expansion.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "fmmpc.h"

namespace fmmpc {

constexpr int MAXP = 20;
constexpr double PI = 3.14159265358979323846;
// -1/(2 pi): kernels multiply by it (FP64 division is a long instruction sequence)
constexpr double NEG_INV_2PI = -0.15915494309189533576888376337251436;

struct Error {
  int code;
  std::string msg;
  Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define FMMPC_CUDA(call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::fmmpc::Error(FMMPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define FMMPC_LAUNCH_CHECK() FMMPC_CUDA(cudaPeekAtLastError())

inline void require(bool ok, const std::string &msg) {
  if (!ok) throw Error(FMMPC_ERR_INVALID, msg);
}

// Device allocation owned by a handle; freed in the handle's destructor.
struct DevPool {
  std::vector<void *> ptrs;
  size_t bytes = 0;
  DevPool() = default;
  DevPool(const DevPool &) = delete;
  DevPool &operator=(const DevPool &) = delete;
  ~DevPool() { release(); }
  void *alloc(size_t nbytes) {
    void *p = nullptr;
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(FMMPC_ERR_OOM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed");
    }
    ptrs.push_back(p);
    bytes += nbytes;
    return p;
  }
  template <typename T>
  T *get(size_t count) {
    return static_cast<T *>(alloc(sizeof(T) * count));
  }
  void release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

// ------------------------------------------------------------------ complex helpers
template <typename R>
struct cpx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  return cpx<R>{a, b};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return cpx<R>{a.re + b.re, a.im + b.im};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return cpx<R>{a.re - b.re, a.im - b.im};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return cpx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return cpx<R>{s * a.re, s * a.im};
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cmac(cpx<R> &acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cinv(cpx<R> a) {
  R d = R(1) / (a.re * a.re + a.im * a.im);
  return cpx<R>{a.re * d, -a.im * d};
}

// ------------------------------------------------------------------ FP64 <-> FP32
// Conversions by the IEEE-754 field layouts on the integer units.  The hardware conversion
// instructions run on the FP64 pipe, which is narrow on this GPU (2 lanes per clock per SM),
// so a kernel that converts once per loaded value can be bound by them.  Values outside the
// range the field arithmetic handles take an out-of-line call to the hardware conversion:
// a real branch, so its FP64 instructions issue only when such a value occurs.
#ifdef __CUDACC__
static __device__ __noinline__ float2 cvt_f64_f32x2_hw(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}
static __device__ __noinline__ double cvt_f32_f64_hw(float f) { return (double)f; }

// x = hi + lo with hi = fl32(x) (round to nearest even) and lo = fl32(x - hi).
__device__ __forceinline__ float2 f64_to_f32x2(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7ffu;
  const uint64_t m = u & 0xfffffffffffffull;
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  if (e >= 923u && e <= 1123u) {  // |x| in [2^-100, 2^101): hi and lo are normal FP32 numbers
    uint32_t f = sign | ((e - 896u) << 23) | (uint32_t)(m >> 29);
    const uint32_t rest = (uint32_t)(m & 0x1fffffffu);  // the 29 bits below FP32 precision
    const bool up = rest > 0x10000000u || (rest == 0x10000000u && (f & 1u));
    f += up ? 1u : 0u;  // a carry out of the mantissa moves into the exponent, as it should
    const int32_t rr = (int32_t)rest - (up ? 0x20000000 : 0);  // x - hi in units of 2^(e - 1075)
    const float mag = __int2float_rn(rr) * 0x1p-29f * __uint_as_float((e - 1046u + 127u) << 23);
    return make_float2(__uint_as_float(f), sign ? -mag : mag);
  }
  if (e == 0 && m == 0) return make_float2(__uint_as_float(sign), __uint_as_float(sign));
  return cvt_f64_f32x2_hw(x);
}

// fl32(x), round to nearest even, as (float)x.
__device__ __forceinline__ float f64_to_f32(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7ffu;
  const uint64_t m = u & 0xfffffffffffffull;
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  if (e >= 897u && e <= 1150u) {  // normal FP32 range; rounding past the largest gives inf
    uint32_t f = sign | ((e - 896u) << 23) | (uint32_t)(m >> 29);
    const uint32_t rest = (uint32_t)(m & 0x1fffffffu);
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if (e == 0 && m == 0) return __uint_as_float(sign);
  return f64_to_f32x2(x).x;
}

// (double)f, exact.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)((uint64_t)u << 32));
  if (e == 0 || e == 0xffu) return cvt_f32_f64_hw(f);
  return __longlong_as_double((long long)(((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                                          ((uint64_t)(u & 0x7fffffu) << 29)));
}

// R(x) for a value loaded as FP64: the field conversion for FP32, the value itself for FP64
template <typename R>
__device__ __forceinline__ R from_f64(double x) {
  if constexpr (sizeof(R) == 4) return f64_to_f32(x);
  else return x;
}
#endif

// ------------------------------------------------------------------ Morton helpers
__host__ __device__ __forceinline__ uint32_t spread_bits16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact_bits16(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0f0f0f0fu;
  x = (x | (x >> 4)) & 0x00ff00ffu;
  x = (x | (x >> 8)) & 0x0000ffffu;
  return x;
}
__host__ __device__ __forceinline__ uint32_t morton_encode(uint32_t ix, uint32_t iy) {
  return spread_bits16(ix) | (spread_bits16(iy) << 1);
}
__host__ __device__ __forceinline__ void morton_decode(uint32_t k, int &ix, int &iy) {
  ix = (int)compact_bits16(k);
  iy = (int)compact_bits16(k >> 1);
}

__host__ __device__ __forceinline__ int64_t level_offset(int l) {
  return ((int64_t(1) << (2 * l)) - 1) / 3;
}
__host__ __device__ __forceinline__ int64_t blevel_offset(int l) {
  return 4 * ((int64_t(1) << l) - 1);
}

// ------------------------------------------------------------------ exact cell geometry
struct GeoDev {
  int n, L, tnum, tden;
};

// Volume cell (level l, Morton c): centre and half-width in units of h/2, origin (x0, y0).
__host__ __device__ __forceinline__ void vol_geom(const GeoDev &g, int l, uint32_t c, int64_t &X,
                                                  int64_t &Y, int64_t &s) {
  int a, b;
  morton_decode(c, a, b);
  int64_t w = g.n >> l;
  X = 2 * a * w + w + 1;
  Y = 2 * b * w + w + 1;
  s = w;
}

// Boundary cell (level l, id = side 2^l + k): the k-th of 2^l equal runs of elements
// along side 0 bottom (x up), 1 right (y up), 2 top (x down), 3 left (y down).  Centre
// and half-width of the circumscribed square in units of h/2^(L+1), origin (x0, y0).
__host__ __device__ __forceinline__ void bnd_geom(const GeoDev &g, int l, uint32_t id, int64_t &X,
                                                  int64_t &Y, int64_t &s) {
  int side = (int)(id >> l);
  int64_t k = id & ((1u << l) - 1u);
  int64_t np1 = g.n + 1, SL = np1 << (g.L + 1);
  int64_t t = (2 * k + 1) * np1 * (int64_t(1) << (g.L - l));
  s = np1 * (int64_t(1) << (g.L - l));
  switch (side) {
    case 0: X = t; Y = 0; break;
    case 1: X = SL; Y = t; break;
    case 2: X = SL - t; Y = SL; break;
    default: X = 0; Y = SL - t; break;
  }
}

// ------------------------------------------------------------------ geometry
struct Geo {
  int n, m, L, lg, p;  // lg = log2(n)
  int tnum, tden;      // theta = tnum / tden
  double x0, y0, side, h, lnh;
  int R;          // P2P stencil radius in leaves (max |offset component|)
  int pad;        // halo of the padded weight image in nodes = R * m
  int npad;       // n + 2 pad
  int NG;         // boundary elements = 4n
  int64_t ncell;  // volume cells, all levels
  int64_t nbcell; // boundary cells, all levels
  int64_t nleaf, nbleaf;
};

// P2P stencil: for each row oy in [-R, R] the contiguous column range [ox0, ox1];
// ox0 > ox1 marks an empty row.
struct Stencil {
  int R;
  int ox0[2 * 16 + 1], ox1[2 * 16 + 1];
  int count;
};

struct Lists {
  int64_t n_m2l = 0, n_p2p = 0, n_m2l_vb = 0, n_p2p_vb = 0;
  int32_t *m2l = nullptr, *p2p = nullptr, *m2l_vb = nullptr, *p2p_vb = nullptr;  // canonical
  // CSR views used by the kernels
  int32_t *m2l_first = nullptr;   // [ncell+1] by global target cell; m2l_src holds sources
  int32_t *m2l_src = nullptr;     // source Morton index at the target's level
  int32_t *vbv_first = nullptr;   // [ncell+1] by volume target: boundary sources (pass B)
  int32_t *vbv_src = nullptr;     // boundary cell id at that level
  int32_t *vbv_cells = nullptr;   // [n_vbv_cells] volume cells whose vbv list is not empty
  int64_t n_vbv_cells = 0;
  int32_t *vbv_slot = nullptr;    // [ncell] index in vbv_cells, -1 for cells without boundary sources
  int32_t *vbb_first = nullptr;   // [nbcell+1] by boundary target: volume sources (pass A)
  int32_t *vbb_src = nullptr;     // volume Morton index at that level
  int32_t *pvb_first = nullptr;   // [nbleaf+1] by boundary leaf: near volume leaves (pass A)
  int32_t *pvb_src = nullptr;
  int32_t *pbv_first = nullptr;   // [nbnear+1] by compacted volume leaf: near boundary leaves
  int32_t *pbv_src = nullptr;
  int32_t *pbv_leaf = nullptr;    // [nbnear] volume leaf Morton index of each compacted row
  int32_t *leaf_bslot = nullptr;  // [nleaf] compacted row of a leaf or -1
  int64_t nbnear = 0;
};

// ------------------------------------------------------------------ cross-file API
// sort_scan.cu
void scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_host,
                        cudaStream_t s, DevPool &tmp);
void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t s,
                    DevPool &tmp);

// tree.cu
struct TreeOut {
  uint32_t *keys;  // natural order
  int32_t *perm;   // Morton position -> natural index
  int32_t *cell_start;
};
void build_tree(const Geo &g, TreeOut &t, cudaStream_t s, DevPool &pool, DevPool &tmp);
void build_lists(const Geo &g, Lists &lists, Stencil &st, cudaStream_t s, DevPool &pool,
                 DevPool &tmp);

}  // namespace fmmpc
