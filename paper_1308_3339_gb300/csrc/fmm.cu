// The preconditioner apply z = P^{-1} r (Sec. 3.2 Fig. f:flow_chart) on the GPU.
//
// Pass A (volume sources w = h^2 r):  P2M at the leaves, M2M up the quadtree (Sec. 5.3
//   items 1-2); M2L from volume cells into the boundary cells, L2L along each side, L2P
//   plus the near field at the collocation points: (V r)(y_m), the right-hand side of
//   Eq. e:ubound with z = 0 on Gamma.  q = S^{-1}(-(V r)|_Gamma) in FP64, or in two-word
//   FP32 in the single-precision forms (Sec. 4.3).
// Pass B: boundary elements carrying q become sources (exact segment multipoles), M2M up
//   the boundary trees; M2L over volume and boundary sources into the volume locals
//   (item 3), L2L down (item 4); the lattice near field (P2P), L2P (item 5) and the
//   closed-form near integrals of the elements complete Eq. e:uinter.
//
// Everything runs in node units with scaled expansions (see common.cuh).  On the uniform
// tree every M2M and L2L is one of a few fixed p x p matrices (child position, side),
// built at set-up from the paper's formulas.  The near field uses the lattice: G between
// two nodes depends only on their integer offset, so P2P is a block convolution of the
// weight image with a table of ln|d| over the stencil of leaf offsets that the dual tree
// traversal produced.
//
// Without stage timing the full apply forks the tensor-core near field, the volume M2L and
// the near-boundary correction onto streams of their own; they overlap the boundary chain
// (collocation values, BEM density, boundary tree) and join before the downward pass.
#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>

#include <set>
#include <type_traits>

#include "handle.cuh"

namespace fmmpc {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// 1/k! for k <= 20, evaluated at compile time (unrolled loops fold it to a constant)
__host__ __device__ constexpr double inv_fact_d(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return 1.0 / f;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ R dev_log(R x) { return log(x); }
template <>
__device__ __forceinline__ float dev_log<float>(float x) { return logf(x); }

// Fixed translation matrices (complex R, row-major [n][k], P = p):
//   vm2m[ch]    volume M2M from child ch (Morton position) to its parent
//   vl2l[ch]    volume L2L from a parent to child ch
//   lvq, lvd, lvp  boundary-element multipole tables per level (described in the struct)
template <typename R>
struct Mats {
  const cpx<R> *vm2m, *vl2l;
  // Multipoles of a boundary element about the centre of its run at every level l (scale
  // n >> l) for a unit single layer (lvq), a unit double layer (lvd) and a unit point source
  // at its midpoint (lvp); level-major, level l at offset 4 P (2n - 2 (n >> l)), then
  // [side][element of the run][P]
  const cpx<R> *lvq, *lvd, *lvp;
};

// ------------------------------------------------------------------ weights
template <typename R>
__global__ void k_weights(int n, int npad, int pad, double h2, int64_t total,
                          const double *__restrict__ r, R *__restrict__ w) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t N = (int64_t)n * n;
  int64_t rhs = t / N, k = t - rhs * N;
  int i = (int)(k % n), j = (int)(k / n);
  w[rhs * npad * (int64_t)npad + (int64_t)(j + pad) * npad + i + pad] = (R)(h2 * r[t]);
}

// ------------------------------------------------------------------ P2M (item 1)
// Mt_0 = sum w_j, Mt_k = -sum w_j zt_j^k / k, zt_j = (z_j - c) / rho_L, by one warp.
template <typename R, int P>
__device__ __forceinline__ void p2m_warp(const R *__restrict__ W, int npad, int pad, int m, uint32_t c,
                                         int lane, cpx<R> (&acc)[P]) {
  int a, b;
  morton_decode(c, a, b);
  const R half = R(0.5) * (m - 1), invm = R(1) / m;
#pragma unroll
  for (int k = 0; k < P; ++k) acc[k] = mk<R>(0, 0);
  for (int t = lane; t < m * m; t += 32) {
    const int i = t % m, j = t / m;
    const R w = W[(int64_t)(b * m + j + pad) * npad + a * m + i + pad];
    const cpx<R> z = mk<R>((i - half) * invm, (j - half) * invm);
    cpx<R> pw = z;
    acc[0].re += w;
#pragma unroll
    for (int k = 1; k < P; ++k) {  // sum w z^k here; the -1/k is applied once per leaf below
      acc[k].re = fma(w, pw.re, acc[k].re);
      acc[k].im = fma(w, pw.im, acc[k].im);
      pw = pw * z;
    }
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const R sk = k == 0 ? R(1) : R(-1) / R(k);
    acc[k].re = sk * warp_sum(acc[k].re);
    acc[k].im = sk * warp_sum(acc[k].im);
  }
}

// parent[n] = sum over 4 children ch, k <= n of T[ch][n][k] child_ch[k]
template <typename R, int P>
__device__ __forceinline__ cpx<R> m2m_row(const cpx<R> *__restrict__ T, const cpx<R> *c0, const cpx<R> *c1,
                                          const cpx<R> *c2, const cpx<R> *c3, int n) {
  cpx<R> acc = mk<R>(0, 0);
  const cpx<R> *ch[4] = {c0, c1, c2, c3};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int k = 0; k <= n; ++k) cmac(acc, T[(q * P + n) * P + k], ch[q][k]);
  return acc;
}

// Sums acc[k] (P <= 16 complex values) over the 16 lanes of a half-warp, transposed: lane c
// of the half ends with the total of acc[c].  The 2P real values, padded to 32, go through a
// butterfly in which each lane keeps half of its values at each of the four steps and adds
// the partner's copy of that half: 30 shuffles where separate trees take 8P.
template <typename R, int P>
__device__ __forceinline__ cpx<R> seg16_sum_coeffs(const cpx<R> (&acc)[P], int c) {
  static_assert(P <= 16, "two values per lane after the butterfly");
  R v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = i < 2 * P ? ((i & 1) ? acc[i >> 1].im : acc[i >> 1].re) : R(0);
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int o = 8 >> st, h = 16 >> st;
    const bool up = (c & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const R keep = up ? v[h + i] : v[i], give = up ? v[i] : v[h + i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  return mk<R>(v[0], v[1]);
}

// k M2M levels (item 2) over the 4^k consecutive (Morton) cells of level l held in
// buf[0 .. 4^k), the first of them cell c0: each level's parents overwrite buf[0 ..) and
// are written to M.  Per output the sum over the four children is split into per-child
// partial sums (at most P terms) run by separate threads, then added in child order.
template <typename R, int P>
__device__ __forceinline__ void m2m_levels_smem(const cpx<R> *sT, cpx<R> (*buf)[P], cpx<R> (*part)[P], cpx<R> *M,
                                                int l, uint32_t c0, int k, int tid, int nthr) {
  for (int lev = 1; lev <= k; ++lev) {
    const int npar = 1 << (2 * (k - lev));
    for (int t = tid; t < 4 * npar * P; t += nthr) {  // (parent, child q, output n)
      const int ch = t / P, q = ch & 3, n = t % P;
      cpx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int kk = 0; kk < P; ++kk)  // fixed trip count: the shared-memory loads go out together
        if (kk <= n) cmac(acc, sT[(q * P + n) * P + kk], buf[ch][kk]);
      part[ch][n] = acc;
    }
    __syncthreads();
    for (int t = tid; t < npar * P; t += nthr) {
      const int pc = t / P, n = t % P;
      const cpx<R> v = part[4 * pc][n] + part[4 * pc + 1][n] + part[4 * pc + 2][n] + part[4 * pc + 3][n];
      buf[pc][n] = v;
      M[(level_offset(l - lev) + (c0 >> (2 * lev)) + pc) * P + n] = v;
    }
    __syncthreads();
  }
}

// The whole upward pass of the volume tree in one launch.  Block (b, rhs) takes the 4x4
// Morton block b of leaves (MS x MS nodes each): P2M (item 1; Mt_0 = sum w_j,
// Mt_k = -sum w_j zt_j^k / k; 16 threads per leaf, each summing every 16th node with all
// its loads issued first, then a shuffle reduction), then M2M (item 2) to the 4 parents and
// to cell b of level L - 2.  Above that, M2M proceeds up to three levels at a time: the
// last of the blocks that complete a Morton group of 4^k cells (an atomic count per group,
// reset by that block) computes the k levels above it.  Any block that does a step
// computes the same sums, so the result does not depend on which block it is.
template <typename R, int P, int MS>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && P <= 10 && MS <= 8) ? 6 : 1) k_upward_tree(Geo g, const R *__restrict__ wpad, const cpx<R> *__restrict__ vm2m,
                                                     cpx<R> *__restrict__ Mv, int *__restrict__ counter, int64_t ncount) {
  // three-level steps need 64 cells in shared memory; two-level steps where that would not fit
  constexpr int NBUF = sizeof(cpx<R>) * P * (4 * P + 128) <= 45000 ? 64 : 16, MAXSTEP = NBUF == 64 ? 3 : 2;
  // z^k of each node position in a leaf (the same for every leaf), where it fits
  constexpr bool ZTAB = sizeof(cpx<R>) * MS * MS * P <= 16384;
  constexpr int ZN = ZTAB ? MS * MS : 1;
  __shared__ cpx<R> sT[4 * P * P], buf[NBUF][P], part[NBUF][P], zt[ZN][P];
  __shared__ int s_last;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rhs = blockIdx.y;
  const uint32_t blk = blockIdx.x;
  for (int i = tid; i < 4 * P * P; i += nthr) sT[i] = vm2m[i];
  cpx<R> *M = Mv + (int64_t)rhs * g.ncell * P;
  {
    constexpr int NP = (MS * MS + 15) / 16;  // nodes per thread
    const int leaf = tid >> 4, c = tid & 15;
    const uint32_t lc = 16 * blk + leaf;
    int a, b;
    morton_decode(lc, a, b);
    const R half = R(0.5) * (MS - 1), invm = R(1) / MS;
    const R *W = wpad + (int64_t)rhs * g.npad * g.npad + (int64_t)(b * MS + g.pad) * g.npad + a * MS + g.pad;
    R w[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) {
      const int pt = c + 16 * e;
      w[e] = pt < MS * MS ? W[(int64_t)(pt / MS) * g.npad + pt % MS] : R(0);
    }
    if (ZTAB) {  // the same chain of products as below, so the same values
      for (int pt = tid; pt < ZN; pt += nthr) {
        const cpx<R> z = mk<R>((pt % MS - half) * invm, (pt / MS - half) * invm);
        cpx<R> pw = z;
        for (int k = 1; k < P; ++k) {
          zt[pt][k] = pw;
          pw = pw * z;
        }
      }
      __syncthreads();
    }
    cpx<R> acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = mk<R>(0, 0);
#pragma unroll
    for (int e = 0; e < NP; ++e) {
      const int pt = c + 16 * e;
      acc[0].re += w[e];
      if (ZTAB) {
        const int ptc = pt < ZN ? pt : 0;  // w[e] is 0 past the leaf
#pragma unroll
        for (int k = 1; k < P; ++k) {
          const cpx<R> zk = zt[ptc][k];
          acc[k].re = fma(w[e], zk.re, acc[k].re);
          acc[k].im = fma(w[e], zk.im, acc[k].im);
        }
      } else {
        const cpx<R> z = mk<R>((pt % MS - half) * invm, (pt / MS - half) * invm);
        cpx<R> pw = z;
#pragma unroll
        for (int k = 1; k < P; ++k) {
          acc[k].re = fma(w[e], pw.re, acc[k].re);
          acc[k].im = fma(w[e], pw.im, acc[k].im);
          pw = pw * z;
        }
      }
    }
    const cpx<R> tot = seg16_sum_coeffs<R, P>(acc, c);  // lane c: coefficient c
    if (c < P) {
      const R sk = c == 0 ? R(1) : R(-1) / R(c);
      const cpx<R> v = mk<R>(sk * tot.re, sk * tot.im);
      buf[leaf][c] = v;
      M[(level_offset(g.L) + lc) * P + c] = v;
    }
  }
  __syncthreads();
  m2m_levels_smem<R, P>(sT, buf, part, M, g.L, 16 * blk, 2, tid, nthr);
  int l = g.L - 2;
  uint32_t cell = blk;
  while (l > 0) {
    const int step = l < MAXSTEP ? l : MAXSTEP, pl = l - step;
    const uint32_t pc = cell >> (2 * step);
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // after the barrier, one fence makes the whole block's writes visible
      int *ctr = counter + (int64_t)rhs * ncount + level_offset(pl) + pc;
      s_last = atomicAdd(ctr, 1) == (1 << (2 * step)) - 1;
      if (s_last) {
        *ctr = 0;  // ready for the next launch
        __threadfence();
      }
    }
    __syncthreads();
    if (!s_last) return;
    const int nch = 1 << (2 * step);
    const uint32_t c0 = pc << (2 * step);
    for (int i = tid; i < nch * P; i += nthr) {
      const R *src = reinterpret_cast<const R *>(M + (level_offset(l) + c0 + i / P) * P + i % P);
      buf[i / P][i % P] = mk<R>(__ldcg(src), __ldcg(src + 1));
    }
    __syncthreads();
    m2m_levels_smem<R, P>(sT, buf, part, M, l, c0, step, tid, nthr);
    l = pl;
    cell = pc;
  }
}

// M2M levels lfrom down to lto (thread per parent coefficient).  One level: a grid of
// threads; several levels: one block that walks them with a barrier between levels.
template <typename R, int P>
__global__ void k_m2m_levels(int lfrom, int lto, int64_t ncell, int nrhs, const cpx<R> *__restrict__ vm2m,
                             cpx<R> *__restrict__ Mv) {
  const bool single = (lfrom == lto);
  for (int l = lfrom; l >= lto; --l) {
    const int64_t nc = int64_t(1) << (2 * l), tasks = nc * P * nrhs;
    const int64_t t0 = single ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x : threadIdx.x;
    const int64_t step = single ? (int64_t)gridDim.x * blockDim.x : blockDim.x;
    for (int64_t t = t0; t < tasks; t += step) {
      const int n = (int)(t % P);
      const int64_t rest = t / P, c = rest % nc;
      const int rhs = (int)(rest / nc);
      cpx<R> *M = Mv + (int64_t)rhs * ncell * P;
      const cpx<R> *ch = M + (level_offset(l + 1) + 4 * c) * P;
      M[(level_offset(l) + c) * P + n] = m2m_row<R, P>(vm2m, ch, ch + P, ch + 2 * P, ch + 3 * P, n);
    }
    if (!single) __syncthreads();
  }
}

// L2L from level l to l+1 for l in [lfrom, lto): child[n] += sum_{k >= n} S[ch][n][k] parent[k].
template <typename R, int P>
__global__ void k_l2l_levels(int lfrom, int lto, int64_t ncell, int nrhs, const cpx<R> *__restrict__ vl2l,
                             cpx<R> *__restrict__ Lv) {
  const bool single = (lto == lfrom + 1);
  for (int l = lfrom; l < lto; ++l) {
    const int64_t nc = int64_t(1) << (2 * (l + 1)), tasks = nc * P * nrhs;
    const int64_t t0 = single ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x : threadIdx.x;
    const int64_t step = single ? (int64_t)gridDim.x * blockDim.x : blockDim.x;
    for (int64_t t = t0; t < tasks; t += step) {
      const int n = (int)(t % P);
      const int64_t rest = t / P, cc = rest % nc;
      const int rhs = (int)(rest / nc);
      cpx<R> *L = Lv + (int64_t)rhs * ncell * P;
      const cpx<R> *Lp = L + (level_offset(l) + (cc >> 2)) * P;
      const cpx<R> *S = vl2l + (int)(cc & 3) * P * P + n * P;
      cpx<R> acc = mk<R>(0, 0);
      for (int k = n; k < P; ++k) cmac(acc, S[k], Lp[k]);
      cpx<R> &dst = L[(level_offset(l + 1) + cc) * P + n];
      dst = dst + acc;
    }
    if (!single) __syncthreads();
  }
}

// ------------------------------------------------------------------ M2L (item 3)
// With zt = (c_target - c_source)/rho (same level), the scaled M2L reads
//   Lt_0 = Mt_0 (log zt + ln rho) + sum_k Mt_k zt^-k
//   Lt_n = ((-1)^n / n!) [ -Mt_0 I_n + sum_k a_k I_{n+k} ],  n >= 1,
// with I_j = (j-1)! zt^-j and a_k = Mt_k / (k-1)!: the paper's M2L formula with
// C(n+k-1, k-1) = (n+k-1)! / ((k-1)! n!) split between source and target.  H collects
// the bracket; the target factor (-1)^n/n! is applied once after the sum over sources.
template <typename R, int P>
__device__ __forceinline__ void m2l_accum(cpx<R> (&H)[P], const cpx<R> *__restrict__ Ms, cpx<R> z,
                                          R lnrho) {
  cpx<R> m[P];
#pragma unroll
  for (int k = 0; k < P; ++k) m[k] = Ms[k];
  const cpx<R> inv = cinv(z);
  cpx<R> I[2 * P];
  I[0] = mk<R>(0, 0);
  I[1] = inv;
#pragma unroll
  for (int j = 2; j < 2 * P; ++j) I[j] = R(j - 1) * (I[j - 1] * inv);
  cpx<R> a[P];
#pragma unroll
  for (int k = 1; k < P; ++k) a[k] = R(inv_fact_d(k - 1)) * m[k];  // m_k / (k-1)!
  const R lz = R(0.5) * dev_log<R>(z.re * z.re + z.im * z.im) + lnrho;
  const R az = atan2(z.im, z.re);
  H[0].re += m[0].re * lz - m[0].im * az;
  H[0].im += m[0].re * az + m[0].im * lz;
#pragma unroll
  for (int k = 1; k < P; ++k) cmac(H[0], a[k], I[k]);
#pragma unroll
  for (int n = 1; n < P; ++n) {
    cmac(H[n], mk<R>(-m[0].re, -m[0].im), I[n]);
#pragma unroll
    for (int k = 1; k < P; ++k) cmac(H[n], a[k], I[n + k]);
  }
}

// warp-reduce H, scale by (-1)^n/n!, then store (add = 0) or accumulate (add = 1)
// Offset between a volume and a boundary cell centre in cell units, d * scale with
// scale = 1 / (rho 2^(L+1)) and d an integer in those fine units.  When the scale is a power
// of two and |d| < 2^24 the FP32 product is exact and equals the FP64 one rounded to FP32,
// so the single-precision forms take it without FP64 instructions (scarce on this GPU).
struct OffsetScale {
  double s64;
  float s32;
  bool exact32;
};
__device__ __forceinline__ OffsetScale offset_scale(int rho, int L) {
  const int64_t v = (int64_t)rho << (L + 1);
  OffsetScale o;
  if ((v & (v - 1)) == 0) {  // 1 / 2^k from the exponent field, no division
    const int k = 63 - __clzll(v);
    o.s64 = __longlong_as_double((long long)(1023 - k) << 52);
    o.exact32 = k < 126;
    o.s32 = o.exact32 ? __int_as_float((127 - k) << 23) : 0.f;
  } else {
    o.s64 = 1.0 / (double)v;
    o.s32 = 0.f;
    o.exact32 = false;
  }
  return o;
}
template <typename R>
__device__ __forceinline__ R scaled_offset(int64_t d, const OffsetScale &o) {
  if (std::is_same<R, float>::value && o.exact32 && d > -(int64_t(1) << 24) && d < (int64_t(1) << 24))
    return (R)((float)d * o.s32);
  return (R)((double)d * o.s64);
}

template <typename R, int P>
__device__ __forceinline__ void m2l_finish(cpx<R> (&H)[P], int lane, cpx<R> *__restrict__ out, int add) {
  R f = 1;
#pragma unroll
  for (int n = 0; n < P; ++n) {
    if (n > 0) f = -f / R(n);
    R re = warp_sum(H[n].re), im = warp_sum(H[n].im);
    if (lane == 0) {
      cpx<R> v = mk(f * re, f * im);
      out[n] = add ? out[n] + v : v;
    }
  }
}

// Volume targets: warp per (cell, rhs).  do_vol: volume sources from the M2L list;
// do_bnd: boundary sources from the volume-boundary list; add: accumulate into L.
// cells (optional): only the listed cells (ntgt of them) instead of all ncell.
template <typename R, int P>
__global__ void k_m2l_vol(GeoDev gd, int64_t ncell, int64_t nbcell, int nrhs, int do_vol, int do_bnd, int add,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                          const int32_t *__restrict__ bfirst, const int32_t *__restrict__ bsrc,
                          const cpx<R> *__restrict__ Mv, const cpx<R> *__restrict__ Mb,
                          cpx<R> *__restrict__ Lv, const int32_t *__restrict__ cells = nullptr,
                          int64_t ntgt = 0) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nt = cells ? ntgt : ncell;
  if (wid >= nt * nrhs) return;
  const int rhs = (int)(wid / nt);
  const int64_t gidx = cells ? (int64_t)cells[wid % nt] : wid % nt;
  int l = 0;
  while (level_offset(l + 1) <= gidx) ++l;
  const uint32_t c = (uint32_t)(gidx - level_offset(l));
  int tx, ty;
  morton_decode(c, tx, ty);
  const int rho = gd.n >> l;
  const R lnrho = dev_log<R>((R)rho);
  cpx<R> H[P];
#pragma unroll
  for (int k = 0; k < P; ++k) H[k] = mk<R>(0, 0);
  if (do_vol) {
    const cpx<R> *M = Mv + (int64_t)rhs * ncell * P + level_offset(l) * P;
    for (int e = first[gidx] + lane; e < first[gidx + 1]; e += 32) {
      const uint32_t s = (uint32_t)src[e];
      int sx, sy;
      morton_decode(s, sx, sy);
      m2l_accum<R, P>(H, M + (int64_t)s * P, mk<R>((R)(tx - sx), (R)(ty - sy)), lnrho);
    }
  }
  if (do_bnd) {
    int64_t X, Y, sw;
    vol_geom(gd, l, c, X, Y, sw);
    X <<= gd.L;
    Y <<= gd.L;
    const OffsetScale scale = offset_scale(rho, gd.L);
    const cpx<R> *MB = Mb + (int64_t)rhs * nbcell * P + blevel_offset(l) * P;
    for (int e = bfirst[gidx] + lane; e < bfirst[gidx + 1]; e += 32) {
      const uint32_t b = (uint32_t)bsrc[e];
      int64_t BX, BY, bs;
      bnd_geom(gd, l, b, BX, BY, bs);
      m2l_accum<R, P>(H, MB + (int64_t)b * P,
                      mk<R>(scaled_offset<R>(X - BX, scale), scaled_offset<R>(Y - BY, scale)), lnrho);
    }
  }
  m2l_finish<R, P>(H, lane, Lv + (int64_t)rhs * ncell * P + gidx * P, add);
}

// Boundary sources added to volume locals, for the cells that have them (cells[0, ntgt)):
// eight lanes per (cell, rhs), four cells per warp, a segmented shuffle reduction, and
// L += (-1)^n/n! H_n (deterministic: no atomics).  The lists average ~8 sources per cell.
// With Lsep the result is written there instead ([rhs][index in cells][P]), for the
// downward pass to add, so that this pass need not wait for the volume M2L.
template <typename R, int P>
__global__ void k_m2l_vbv(GeoDev gd, int64_t ncell, int64_t nbcell, int nrhs, const int32_t *__restrict__ bfirst,
                          const int32_t *__restrict__ bsrc, const cpx<R> *__restrict__ Mb, cpx<R> *__restrict__ Lv,
                          const int32_t *__restrict__ cells, int64_t ntgt, cpx<R> *__restrict__ Lsep = nullptr) {
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int sub = threadIdx.x & 7;
  const bool active = grp < ntgt * nrhs;
  const int64_t gg = active ? grp : 0;
  const int rhs = (int)(gg / ntgt);
  const int64_t gidx = cells[gg % ntgt];
  int l = 0;
  while (level_offset(l + 1) <= gidx) ++l;
  const uint32_t c = (uint32_t)(gidx - level_offset(l));
  const int rho = gd.n >> l;
  const R lnrho = dev_log<R>((R)rho);
  cpx<R> H[P];
#pragma unroll
  for (int k = 0; k < P; ++k) H[k] = mk<R>(0, 0);
  if (active) {
    int64_t X, Y, sw;
    vol_geom(gd, l, c, X, Y, sw);
    X <<= gd.L;
    Y <<= gd.L;
    const OffsetScale scale = offset_scale(rho, gd.L);
    const cpx<R> *MB = Mb + (int64_t)rhs * nbcell * P + blevel_offset(l) * P;
    for (int e = bfirst[gidx] + sub; e < bfirst[gidx + 1]; e += 8) {
      const uint32_t b = (uint32_t)bsrc[e];
      int64_t BX, BY, bs;
      bnd_geom(gd, l, b, BX, BY, bs);
      m2l_accum<R, P>(H, MB + (int64_t)b * P,
                      mk<R>(scaled_offset<R>(X - BX, scale), scaled_offset<R>(Y - BY, scale)), lnrho);
    }
  }
  R f = 1;
  cpx<R> *out = Lsep ? Lsep + ((int64_t)rhs * ntgt + gg % ntgt) * P : Lv + (int64_t)rhs * ncell * P + gidx * P;
#pragma unroll
  for (int n = 0; n < P; ++n) {
    if (n > 0) f = -f / R(n);
    R re = H[n].re, im = H[n].im;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (active && sub == 0) out[n] = Lsep ? mk(f * re, f * im) : out[n] + mk(f * re, f * im);
  }
}

// Boundary targets (pass A): warp per (boundary cell, rhs); volume sources.
template <typename R, int P>
__global__ void k_m2l_bnd(GeoDev gd, int64_t ncell, int64_t nbcell, int nrhs,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                          const cpx<R> *__restrict__ Mv, cpx<R> *__restrict__ Lb, double lnh) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nbcell * nrhs) return;
  const int rhs = (int)(wid / nbcell);
  const int64_t gb = wid % nbcell;
  int l = 0;
  while (blevel_offset(l + 1) <= gb) ++l;
  const uint32_t b = (uint32_t)(gb - blevel_offset(l));
  const int rho = gd.n >> l;
  const R lnrho = dev_log<R>((R)rho);
  int64_t BX, BY, bs;
  bnd_geom(gd, l, b, BX, BY, bs);
  const OffsetScale scale = offset_scale(rho, gd.L);
  cpx<R> H[P];
#pragma unroll
  for (int k = 0; k < P; ++k) H[k] = mk<R>(0, 0);
  const cpx<R> *M = Mv + (int64_t)rhs * ncell * P + level_offset(l) * P;
  for (int e = first[gb] + lane; e < first[gb + 1]; e += 32) {
    const uint32_t v = (uint32_t)src[e];
    int64_t X, Y, sw;
    vol_geom(gd, l, v, X, Y, sw);
    X <<= gd.L;
    Y <<= gd.L;
    m2l_accum<R, P>(H, M + (int64_t)v * P,
                    mk<R>(scaled_offset<R>(BX - X, scale), scaled_offset<R>(BY - Y, scale)), lnrho);
  }
  m2l_finish<R, P>(H, lane, Lb + (int64_t)rhs * nbcell * P + gb * P, 0);
  // the four side roots also take the ln h part of G times the total volume weight
  if (gb < 4 && lane == 0)
    Lb[(int64_t)rhs * nbcell * P + gb * P].re += (R)(lnh * (double)Mv[(int64_t)rhs * ncell * P].re);
}

// ------------------------------------------------------------------ root constants
// The ln h part of G times the total weight, added to the root local expansions.
// mode 0: boundary roots += ln h W_vol (pass A); 1: volume root += ln h W_vol;
// 2: volume root += ln h (W_vol + W_bnd).
template <typename R>
__global__ void k_root_const(int p, int64_t ncell, int64_t nbcell, int nrhs, double lnh, int mode,
                             const cpx<R> *__restrict__ Mv, const cpx<R> *__restrict__ Mb,
                             cpx<R> *__restrict__ Lv, cpx<R> *__restrict__ Lb) {
  for (int rhs = threadIdx.x; rhs < nrhs; rhs += blockDim.x) {
    double W = (double)Mv[(int64_t)rhs * ncell * p].re;
    if (mode == 0) {
      for (int s = 0; s < 4; ++s) Lb[(int64_t)rhs * nbcell * p + (int64_t)s * p].re += (R)(lnh * W);
    } else {
      if (mode == 2)
        for (int s = 0; s < 4; ++s) W += (double)Mb[(int64_t)rhs * nbcell * p + (int64_t)s * p].re;
      Lv[(int64_t)rhs * ncell * p].re += (R)(lnh * W);
    }
  }
}

// ------------------------------------------------------------------ boundary geometry
// Along-side coordinate u and signed normal offset d of node coordinates (x, y): for an
// element starting at arclength t_a, s1 = t_a - u and d = (x - a).n_outward (Sec. 4.3).
__device__ __forceinline__ void side_coords(int side, int np1, int x, int y, int &u, int &d) {
  switch (side) {
    case 0: u = x; d = -y; break;
    case 1: u = y; d = x - np1; break;
    case 2: u = np1 - x; d = y - np1; break;
    default: u = np1 - y; d = -x; break;
  }
}

// Multipoles of every boundary cell at every level in one launch,
// Mt_k = sum_e (q_e qscale Bq_l[e][k] + qd_e dsgn Bd_l[e][k]) over the elements e of the cell,
// with the level tables of Mats (element single layer, double layer, or point source at
// the midpoint; [side][element of the cell][p] per level); HQ, HD say whether q and qd are
// given.  Work units are runs of at most 16 consecutive elements of one cell (a level's
// units are consecutive in element order); a block of 16 x 16 threads takes 16 units of
// one level, converts their element weights once each into shared memory, and thread
// (unit, k) accumulates coefficient k over its unit's elements, the table loads of a batch
// of eight issued before they are added.  The units of a cell then meet in shared memory in
// a fixed order.  Cells of more than 256 elements (the Lc coarse levels) span several
// blocks: each block writes its partial to part, and the last block of the cell to arrive
// (an atomic count per cell, reset by that block) adds the partials in order.  So fine cells
// share blocks, and no thread waits on more than 16 elements' loads at any level.
constexpr int BUP_CHUNK = 256;  // elements per block at most (16 units of 16)
template <typename R, int P, bool HQ, bool HD>
__global__ void __launch_bounds__(256) k_bnd_up_lv(Geo g, int nrhs, int Lc, const double *__restrict__ q,
                                                   const cpx<R> *__restrict__ Bq, R qscale,
                                                   const double *__restrict__ qd, const cpx<R> *__restrict__ Bd,
                                                   R dsgn, cpx<R> *__restrict__ Mb, cpx<R> *__restrict__ part,
                                                   int *__restrict__ cnt) {
  static_assert(P <= 16, "one coefficient slot per thread");
  __shared__ R sre[16][17], sim[16][17];
  __shared__ R swq[BUP_CHUNK], swd[BUP_CHUNK];  // the block's element weights, converted once
  __shared__ int s_last;
  const int rhs = blockIdx.y;
  const int ul = threadIdx.x >> 4, k = threadIdx.x & 15;
  const int n = g.n;
  // level of this block, and its first unit in the level
  int l = 0, bi = (int)blockIdx.x;
  for (;;) {
    const int len = n >> l, upc = len > 16 ? len / 16 : 1;
    const int nb = (((4 << l) * upc) + 15) / 16;
    if (bi < nb || l == g.L) break;
    bi -= nb;
    ++l;
  }
  const int len = n >> l, upc = len > 16 ? len / 16 : 1, ue = len < 16 ? len : 16;
  const int units = (4 << l) * upc, u0 = bi * 16;
  const int64_t E0 = (int64_t)u0 * ue;  // first element of the block (level element order)
  const int nel = min(16, units - u0) * ue;
  const int64_t rbase = (int64_t)rhs * g.NG;
  if ((int)threadIdx.x < nel) {
    if (HQ) swq[threadIdx.x] = from_f64<R>(q[rbase + E0 + threadIdx.x]) * qscale;
    if (HD) swd[threadIdx.x] = from_f64<R>(qd[rbase + E0 + threadIdx.x]) * dsgn;
  }
  __syncthreads();
  const int u = u0 + ul;
  R are = 0, aim = 0;
  if (k < P && u < units) {
    const int64_t cellid = u / upc;            // id = side 2^l + run
    const int side = (int)(cellid >> l);
    const int e1 = (u % upc) * ue;             // first element of the unit within its cell
    const int64_t toff = (int64_t)4 * P * (2 * n - 2 * len) + ((int64_t)side * len + e1) * P + k;
    const int s0 = ul * ue;                     // the unit's weights in shared memory
    constexpr int U = 8;
#pragma unroll
    for (int b0 = 0; b0 < 16; b0 += U) {
      if (b0 >= ue) break;
      cpx<R> b1[U], b2[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        if (HQ) b1[i] = b0 + i < ue ? Bq[toff + (int64_t)(b0 + i) * P] : mk<R>(0, 0);
        if (HD) b2[i] = b0 + i < ue ? Bd[toff + (int64_t)(b0 + i) * P] : mk<R>(0, 0);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) {
        if (b0 + i < ue) {
          if (HQ) {
            const R w1 = swq[s0 + b0 + i];
            are = fma(w1, b1[i].re, are);
            aim = fma(w1, b1[i].im, aim);
          }
          if (HD) {
            const R w2 = swd[s0 + b0 + i];
            are = fma(w2, b2[i].re, are);
            aim = fma(w2, b2[i].im, aim);
          }
        }
      }
    }
  }
  sre[ul][k] = are;
  sim[ul][k] = aim;
  __syncthreads();
  if (upc <= 16) {  // whole cells in this block: 16 / upc of them
    const int cb = threadIdx.x >> 4, ncb = 16 / upc;
    const int64_t cellid = (int64_t)u0 / upc + cb;
    if (cb < ncb && k < P && cellid < (4 << l)) {
      R re = 0, im = 0;
      for (int j = 0; j < upc; ++j) {
        re += sre[cb * upc + j][k];
        im += sim[cb * upc + j][k];
      }
      Mb[((int64_t)rhs * g.nbcell + blevel_offset(l) + cellid) * P + k] = mk<R>(re, im);
    }
    return;  // block-uniform
  }
  // a coarse cell: this block's partial, then the cell's last block adds them in order
  const int nch = upc / 16, chunk = (u0 % upc) / 16;
  const int64_t cell = blevel_offset(l) + u0 / upc;
  if (threadIdx.x < P) {
    R re = 0, im = 0;
    for (int j = 0; j < 16; ++j) {
      re += sre[j][threadIdx.x];
      im += sim[j][threadIdx.x];
    }
    part[((int64_t)rhs * gridDim.x + blockIdx.x) * P + threadIdx.x] = mk<R>(re, im);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int *ct = cnt + (int64_t)rhs * blevel_offset(Lc) + cell;
    s_last = atomicAdd(ct, 1) == nch - 1;
    if (s_last) *ct = 0;  // ready for the next launch
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < P) {
    const cpx<R> *pp = part + ((int64_t)rhs * gridDim.x + blockIdx.x - chunk) * P + threadIdx.x;
    R sr = 0, si = 0;
    for (int c = 0; c < nch; ++c) {
      sr += __ldcg(&pp[(int64_t)c * P].re);
      si += __ldcg(&pp[(int64_t)c * P].im);
    }
    Mb[((int64_t)rhs * g.nbcell + cell) * P + threadIdx.x] = mk<R>(sr, si);
  }
}

// Blocks of k_bnd_up_lv for an n-side grid with L + 1 boundary levels.
inline int64_t bup_blocks(int n, int L) {
  int64_t nb = 0;
  for (int l = 0; l <= L; ++l) {
    const int len = n >> l, upc = len > 16 ? len / 16 : 1;
    nb += (((int64_t)(4 << l) * upc) + 15) / 16;
  }
  return nb;
}


// ------------------------------------------------------------------ collocation points
// Set-up for the single-precision forms: the near-field log kernel between each collocation
// point and the nodes of its near volume leaves, formed in FP64 and stored FP32.  Warp per
// point; layout [boundary leaf: pfirst m m^2][point in leaf][near leaf][node].
__global__ void k_colloc_mat(Geo g, const int32_t *__restrict__ pfirst, const int32_t *__restrict__ psrc,
                             float *__restrict__ Kc) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)g.NG) return;
  const int ge = (int)wid, n = g.n, m = g.m, L = g.L;
  const int side = ge / n, along = ge % n;
  const int64_t bl = ((int64_t)side << L) + along / m;
  const int64_t numc = (2 * (int64_t)along + 1) * (n + 1);
  const int c_near = pfirst[bl + 1] - pfirst[bl];
  const int64_t kbase = ((int64_t)pfirst[bl] * m + (int64_t)(along % m) * c_near) * (m * m);
  for (int e0 = pfirst[bl]; e0 < pfirst[bl + 1]; ++e0) {
    int a, b;
    morton_decode((uint32_t)psrc[e0], a, b);
    float *kr = Kc + kbase + (int64_t)(e0 - pfirst[bl]) * (m * m);
    for (int t = lane; t < m * m; t += 32) {
      const int i = a * m + t % m, j = b * m + t / m;
      int u, d;
      side_coords(side, n + 1, i + 1, j + 1, u, d);
      const double ds = (double)(numc - 2 * (int64_t)u * n) / (2.0 * n);
      kr[t] = (float)(0.5 * log(ds * ds + (double)d * (double)d));
    }
  }
}


// (V r)(y_m) = -(1/2pi)[ Re sum_n Lt_n zt^n  +  sum_{near nodes} w_j ln|y_m - x_j| ].
// Warp per (collocation point, rhs); requires L < 32.  mode 0: both sums; mode 1: the near
// sum alone, into vnear (it needs only the weights, so it can run beside the volume
// upward pass); mode 2: the far sum, added to the near sum read from vnear.
template <typename R>
__global__ void k_colloc(Geo g, int nrhs, const R *__restrict__ wpad, const cpx<R> *__restrict__ Lb,
                         const int32_t *__restrict__ pfirst, const int32_t *__restrict__ psrc,
                         double *__restrict__ vcol, const float *__restrict__ Kc, float *__restrict__ vt_hi,
                         float *__restrict__ vt_lo, int mode, R *__restrict__ vnear) {
  // block (rhs, along): warp w takes the collocation point `along` of side w
  __shared__ double sv[4];
  const int lane = threadIdx.x & 31;
  const int rhs = (int)(blockIdx.x / g.n), along = (int)(blockIdx.x % g.n), side = threadIdx.x >> 5;
  const int n = g.n, m = g.m, L = g.L, p = g.p;
  const int ge = side * n + along;
  const int64_t bl = ((int64_t)side << L) + along / m;
  const R *W = wpad + (int64_t)rhs * g.npad * g.npad;
  const R inv2n = R(1) / (R)(2 * n);
  const int64_t numc = (2 * (int64_t)along + 1) * (n + 1);
  R acc = 0;
  // precomputed (single-precision forms): Kc[(pfirst m + ip c) m^2 + el m^2 + t] = ln|y - x_t|
  const int c_near = pfirst[bl + 1] - pfirst[bl];
  const int64_t kbase = ((int64_t)pfirst[bl] * m + (int64_t)(along % m) * c_near) * (m * m);
  bool done_near = mode == 2;
  if (mode == 2) acc = vnear[(int64_t)rhs * g.NG + ge];
  if constexpr (std::is_same<R, float>::value) {
    if (!done_near && Kc && m == 8 && (g.pad & 3) == 0 && (g.npad & 3) == 0) {
      // 16 lanes per near leaf, 4 consecutive nodes of a leaf row per lane (float4)
      const float4 *k4 = reinterpret_cast<const float4 *>(Kc + kbase);
#pragma unroll 4
      for (int it = lane; it < c_near * 16; it += 32) {
        const int el = it >> 4, t4 = it & 15;
        int a, b;
        morton_decode((uint32_t)psrc[pfirst[bl] + el], a, b);
        const int row = b * 8 + (t4 >> 1), col = a * 8 + (t4 & 1) * 4;
        const float4 wv = *reinterpret_cast<const float4 *>(W + (int64_t)(row + g.pad) * g.npad + col + g.pad);
        const float4 kv = k4[it];
        acc += wv.x * kv.x + wv.y * kv.y + wv.z * kv.z + wv.w * kv.w;
      }
      done_near = true;
    }
  }
  if (!done_near)
  for (int e0 = pfirst[bl]; e0 < pfirst[bl + 1]; ++e0) {
    int a, b;
    morton_decode((uint32_t)psrc[e0], a, b);
    if (Kc) {
      const float *kr = Kc + kbase + (int64_t)(e0 - pfirst[bl]) * (m * m);
      for (int t = lane; t < m * m; t += 32)
        acc += W[(int64_t)(b * m + t / m + g.pad) * g.npad + a * m + t % m + g.pad] * (R)kr[t];
      continue;
    }
    for (int t = lane; t < m * m; t += 32) {
      const int i = a * m + t % m, j = b * m + t / m;
      int u, d;
      side_coords(side, n + 1, i + 1, j + 1, u, d);
      // (y_e - x) along the side = ((2 along + 1)(n + 1) - 2 u n) / (2n), exact numerator
      const R ds = (R)(numc - 2 * (int64_t)u * n) * inv2n;
      acc += W[(int64_t)(j + g.pad) * g.npad + i + g.pad] * (R(0.5) * dev_log<R>(ds * ds + (R)d * (R)d));
    }
  }
  if (mode != 2) acc = warp_sum(acc);
  if (mode == 1) {
    if (lane == 0) vnear[(int64_t)rhs * g.NG + ge] = acc;
    return;  // warp-uniform; mode 1 takes no barrier below
  }
  // far field: the local expansion of every ancestor run evaluated at y (L2L re-centring
  // is exact, so this equals pushing the locals down to the leaf run and evaluating there)
  R far = 0;
  if (lane <= L) {
    const int l = lane, nl = n >> l;
    const int64_t id = ((int64_t)side << l) + along / nl;
    // offset of the point from the run centre, in run units: (n+1)/n (j + 1/2 - nl/2) / nl
    const R off = (R)(n + 1) * ((R)(along % nl) + R(0.5) - R(0.5) * (R)nl) / ((R)n * (R)nl);
    const R ex = (side == 0) ? R(1) : (side == 2 ? R(-1) : R(0));
    const R ey = (side == 1) ? R(1) : (side == 3 ? R(-1) : R(0));
    const cpx<R> z = mk<R>(off * ex, off * ey);
    const cpx<R> *Lc = Lb + (int64_t)rhs * g.nbcell * p + (blevel_offset(l) + id) * p;
    cpx<R> v = mk<R>(0, 0);
    for (int kk = p - 1; kk >= 0; --kk) v = v * z + Lc[kk];
    far = v.re;
  }
  far = warp_sum(far);
  const double v = ((double)acc + (double)far) * NEG_INV_2PI;
  if (lane == 0) {
    vcol[(int64_t)rhs * g.NG + ge] = v;
    sv[side] = v;
  }
  if (vt_hi) {
    // the side DFT of the four values (as k_bem_vt) as FP32 hi + lo words for the BEM apply
    __syncthreads();
    if (threadIdx.x < 4) {
      const int j = threadIdx.x;
      const double o = j == 0 ? (sv[0] + sv[2]) + (sv[1] + sv[3])
                     : j == 1 ? (sv[0] + sv[2]) - (sv[1] + sv[3])
                     : j == 2 ? sv[0] - sv[2] : sv[1] - sv[3];
      const float hi = (float)o;
      vt_hi[(int64_t)rhs * g.NG + j * n + along] = hi;
      vt_lo[(int64_t)rhs * g.NG + j * n + along] = (float)(o - (double)hi);
    }
  }
}

// ------------------------------------------------------------------ BEM solve (FP64)
// q = -S^{-1} (V r)|_Gamma with the inverse formed at set-up.  Rotating the square by 90
// degrees maps element (side s, index k) to (s+1, k), so S and its inverse are block
// circulant in the four sides: q_s = -sum_d C_d v_{s+d}, C_d the blocks of the first block
// row.  A 4-point DFT over the side index diagonalises this: with
//   C^0 = C0+C1+C2+C3, C^2 = C0-C1+C2-C3, A = C0-C2, B = C1-C3 (stored at set-up) and
//   v^0 = v0+v1+v2+v3, v^2 = v0-v1+v2-v3, a = v0-v2, b = v1-v3,
// P0 = C^0 v^0, P2 = C^2 v^2, R + iI = (A + iB)(a - ib), and
//   q0 = -(P0+P2+2R)/4, q1 = -(P0-P2-2I)/4, q2 = -(P0+P2-2R)/4, q3 = -(P0-P2+2I)/4:
// 6 n^2 FP64 multiply-adds instead of 16 n^2 (FP64 is the bound on this part).

// The boundary data term of Eq. e:ubound moved to the left: vcol_m -= (1/2 g_m + (K g)_m)
// at every collocation point, K_mk = int_k dG/dn_y(y_m, y) dGamma = (1/2pi) atan2(l d,
// d^2 + s1 s2) (zero on the point's own side), so that the BEM solve q = S^{-1}(-vcol) gives
// S q = (1/2 I + K) g - (V f)|_Gamma.  Block per (collocation point, rhs), FP64.
__global__ void __launch_bounds__(256) k_dl_colloc(int n, int nrhs, const double *__restrict__ gdat,
                                                   double *__restrict__ vcol) {
  __shared__ double red[8];
  const int mrow = blockIdx.x, rhs = blockIdx.y, NG = 4 * n;
  const double ell = (n + 1.0) / n, np1 = n + 1.0;
  const int sm = mrow / n, km = mrow % n;
  const double tm = (km + 0.5) * ell;
  double x, y;
  switch (sm) {
    case 0: x = tm; y = 0; break;
    case 1: x = np1; y = tm; break;
    case 2: x = np1 - tm; y = np1; break;
    default: x = 0; y = np1 - tm; break;
  }
  const double *gr = gdat + (int64_t)rhs * NG;
  double acc = 0.0;
  for (int k = threadIdx.x; k < NG; k += blockDim.x) {
    const int sk = k / n, kk = k % n;
    if (sk == sm) continue;
    double u, d;
    switch (sk) {
      case 0: u = x; d = -y; break;
      case 1: u = y; d = x - np1; break;
      case 2: u = np1 - x; d = y - np1; break;
      default: u = np1 - y; d = -x; break;
    }
    const double s1 = kk * ell - u, s2 = s1 + ell;
    acc += gr[k] * atan2(ell * d, d * d + s1 * s2);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    vcol[(int64_t)rhs * NG + mrow] -= 0.5 * gr[mrow] + t / (2.0 * PI);
  }
}

// vt[rhs] = [v^0 | v^2 | a | b] from vcol[rhs] = [v0 | v1 | v2 | v3]
__global__ void k_bem_vt(int n, int nrhs, const double *__restrict__ vcol, double *__restrict__ vt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrhs * n) return;
  const int64_t rr = t / n;
  const int k = (int)(t % n);
  const double *v = vcol + rr * 4 * n;
  const double v0 = v[k], v1 = v[n + k], v2 = v[2 * n + k], v3 = v[3 * n + k];
  double *o = vt + rr * 4 * n;
  o[k] = (v0 + v2) + (v1 + v3);
  o[n + k] = (v0 + v2) - (v1 + v3);
  o[2 * n + k] = v0 - v2;
  o[3 * n + k] = v1 - v3;
}

// Block per row m of the transformed first block row T[m] = [C^0 | C^2 | A | B][m].
__global__ void __launch_bounds__(256) k_bem_apply(int n, int nrhs, const double *__restrict__ T,
                                                   const double *__restrict__ vt, double *__restrict__ q) {
  __shared__ double red[8][4];
  const int mrow = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int NG = 4 * n;
  const double *Tr = T + (int64_t)mrow * NG;
  for (int rr = 0; rr < nrhs; ++rr) {
    const double *v = vt + (int64_t)rr * NG;
    double p0 = 0.0, p2 = 0.0, re = 0.0, im = 0.0;
    for (int k = tid; k < n; k += 256) {
      const double c0 = Tr[k], c2 = Tr[n + k], ca = Tr[2 * n + k], cb = Tr[3 * n + k];
      const double a = v[2 * n + k], b = v[3 * n + k];
      p0 = fma(c0, v[k], p0);
      p2 = fma(c2, v[n + k], p2);
      re = fma(ca, a, fma(cb, b, re));
      im = fma(cb, a, fma(-ca, b, im));
    }
    double acc[4] = {p0, p2, re, im};
#pragma unroll
    for (int sg = 0; sg < 4; ++sg) {
      const double x = warp_sum(acc[sg]);
      if (lane == 0) red[w][sg] = x;
    }
    __syncthreads();
    if (tid == 0) {
      double P0 = 0.0, P2 = 0.0, R = 0.0, I = 0.0;
      for (int ww = 0; ww < 8; ++ww) {
        P0 += red[ww][0];
        P2 += red[ww][1];
        R += red[ww][2];
        I += red[ww][3];
      }
      double *qr = q + (int64_t)rr * NG;
      qr[mrow] = -0.25 * (P0 + P2 + 2.0 * R);
      qr[n + mrow] = -0.25 * (P0 - P2 - 2.0 * I);
      qr[2 * n + mrow] = -0.25 * (P0 + P2 - 2.0 * R);
      qr[3 * n + mrow] = -0.25 * (P0 - P2 + 2.0 * I);
    }
    __syncthreads();
  }
}

// Two-word FP32 arithmetic for the BEM apply of the single-precision forms (FP64 is scarce
// on this GPU): a value x is carried as hi + lo, hi = fl32(x), lo = fl32(x - hi).
// s + c += p with Knuth's TwoSum (the rounding error of s + p goes into c).
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float p) {
  const float t = s + p, bb = t - s;
  c += (s - (t - bb)) + (p - bb);
  s = t;
}
// s + c += (ah + al)(bh + bl): the product ah bh split exactly by an FMA, the cross terms
// into c (the dot product of Ogita, Rump and Oishi, "Dot2", with the operands' low words).
__device__ __forceinline__ void dot2_mac(float &s, float &c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = fmaf(ah, bh, -p);
  two_sum_acc(s, c, p);
  c = fmaf(al, bh, fmaf(ah, bl, c + e));
}

// The BEM apply of k_bem_apply in two-word FP32 arithmetic: two warps per row m of
// T = [C^0 | C^2 | A | B], each half of its columns (two rows per block), RB right-hand sides
// per pass over it.  A lane takes four consecutive columns at a time (16-byte loads of the
// four blocks, hi and lo) and two such steps at once, so that a row's loads are in flight
// together and the pass is a sweep over T at memory speed rather than a chain of load round
// trips.  The partial two-word sums are combined with TwoSum over the warp's lanes, then
// over the row's two warps, and converted to FP64 once per row and right-hand side.  n is a
// multiple of 8 and the rows start 16-byte aligned.
constexpr int BEM_ROWS = 2;  // rows per block, two warps each
template <int RB>
__global__ void __launch_bounds__(64 * BEM_ROWS) k_bem_apply_f2(int n, int nrhs, const float *__restrict__ Th,
                                                              const float *__restrict__ Tl, const float *__restrict__ vh,
                                                              const float *__restrict__ vl, double *__restrict__ q) {
  __shared__ float xs[BEM_ROWS][RB][4], xc[BEM_ROWS][RB][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, rb = w >> 1, hw = w & 1;
  const int mrow = blockIdx.x * BEM_ROWS + rb;
  const bool live = mrow < n;  // block-uniform for the barrier below: n is a multiple of BEM_ROWS
  const int NG = 4 * n, n4 = n >> 2, kbeg = hw * (n4 >> 1), kend = kbeg + (n4 >> 1);
  const float4 *th = reinterpret_cast<const float4 *>(Th + (int64_t)mrow * NG);
  const float4 *tl = reinterpret_cast<const float4 *>(Tl + (int64_t)mrow * NG);
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    float sa[RB][4], ca[RB][4];
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
      for (int g = 0; g < 4; ++g) sa[j][g] = ca[j][g] = 0.f;
#pragma unroll 2
    for (int k4 = kbeg + lane; live && k4 < kend; k4 += 32) {
      const float4 c0h = th[k4], c2h = th[n4 + k4], cah = th[2 * n4 + k4], cbh = th[3 * n4 + k4];
      const float4 c0l = tl[k4], c2l = tl[n4 + k4], cal = tl[2 * n4 + k4], cbl = tl[3 * n4 + k4];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        if (r0 + j < nrhs) {
          const float4 *xh = reinterpret_cast<const float4 *>(vh + (int64_t)(r0 + j) * NG);
          const float4 *xl = reinterpret_cast<const float4 *>(vl + (int64_t)(r0 + j) * NG);
          const float4 v0h = xh[k4], v2h = xh[n4 + k4], ah = xh[2 * n4 + k4], bh = xh[3 * n4 + k4];
          const float4 v0l = xl[k4], v2l = xl[n4 + k4], al = xl[2 * n4 + k4], bl = xl[3 * n4 + k4];
          const float c0h_[4] = {c0h.x, c0h.y, c0h.z, c0h.w}, c0l_[4] = {c0l.x, c0l.y, c0l.z, c0l.w};
          const float c2h_[4] = {c2h.x, c2h.y, c2h.z, c2h.w}, c2l_[4] = {c2l.x, c2l.y, c2l.z, c2l.w};
          const float cah_[4] = {cah.x, cah.y, cah.z, cah.w}, cal_[4] = {cal.x, cal.y, cal.z, cal.w};
          const float cbh_[4] = {cbh.x, cbh.y, cbh.z, cbh.w}, cbl_[4] = {cbl.x, cbl.y, cbl.z, cbl.w};
          const float v0h_[4] = {v0h.x, v0h.y, v0h.z, v0h.w}, v0l_[4] = {v0l.x, v0l.y, v0l.z, v0l.w};
          const float v2h_[4] = {v2h.x, v2h.y, v2h.z, v2h.w}, v2l_[4] = {v2l.x, v2l.y, v2l.z, v2l.w};
          const float ah_[4] = {ah.x, ah.y, ah.z, ah.w}, al_[4] = {al.x, al.y, al.z, al.w};
          const float bh_[4] = {bh.x, bh.y, bh.z, bh.w}, bl_[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            dot2_mac(sa[j][0], ca[j][0], c0h_[c], c0l_[c], v0h_[c], v0l_[c]);
            dot2_mac(sa[j][1], ca[j][1], c2h_[c], c2l_[c], v2h_[c], v2l_[c]);
            dot2_mac(sa[j][2], ca[j][2], cah_[c], cal_[c], ah_[c], al_[c]);  // re = A a + B b
            dot2_mac(sa[j][2], ca[j][2], cbh_[c], cbl_[c], bh_[c], bl_[c]);
            dot2_mac(sa[j][3], ca[j][3], cbh_[c], cbl_[c], ah_[c], al_[c]);  // im = B a - A b
            dot2_mac(sa[j][3], ca[j][3], -cah_[c], -cal_[c], bh_[c], bl_[c]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
      for (int g = 0; g < 4; ++g) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float s2 = __shfl_xor_sync(0xffffffffu, sa[j][g], o), c2 = __shfl_xor_sync(0xffffffffu, ca[j][g], o);
          two_sum_acc(sa[j][g], ca[j][g], s2);
          ca[j][g] += c2;
        }
        if (hw == 1 && lane == 0) {
          xs[rb][j][g] = sa[j][g];
          xc[rb][j][g] = ca[j][g];
        }
      }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      double tot[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float s0 = sa[j][g], c0 = ca[j][g];  // the first half's sums (lane 0 of warp hw = 0)
        two_sum_acc(s0, c0, xs[rb][j][g]);
        c0 += xc[rb][j][g];
        tot[g] = (double)s0 + (double)c0;
      }
      if (hw == 0 && lane == 0 && live && r0 + j < nrhs) {
        const double P0 = tot[0], P2 = tot[1], R = tot[2], I = tot[3];
        double *qr = q + (int64_t)(r0 + j) * NG;
        qr[mrow] = -0.25 * (P0 + P2 + 2.0 * R);
        qr[n + mrow] = -0.25 * (P0 - P2 - 2.0 * I);
        qr[2 * n + mrow] = -0.25 * (P0 + P2 - 2.0 * R);
        qr[3 * n + mrow] = -0.25 * (P0 - P2 + 2.0 * I);
      }
    }
    __syncthreads();  // xs, xc are rewritten by the next pass
  }
}

// ------------------------------------------------------------------ near boundary field
// int over an element of ln|x - y| ds (node units), stable closed form:
// with s1 = (a - x).t, s2 = s1 + l, d = (x - a).n, A_i = s_i^2 + d^2,
// = 1/2 [ l ln A2 + s1 log1p(l (s1 + s2) / A1) ] - l + d atan2(l d, d^2 + s1 s2).
template <typename R>
__device__ __forceinline__ R seg_log_int(R s1, R ell, R d) {
  const R s2 = s1 + ell;
  const R A1 = s1 * s1 + d * d, A2 = s2 * s2 + d * d;
  R v = R(0.5) * (ell * dev_log<R>(A2) + s1 * log1p(ell * (s1 + s2) / A1)) - ell;
  if (d != R(0)) v += d * atan2(ell * d, d * d + s1 * s2);
  return v;
}

// Block of 256 per (volume leaf next to the boundary, rhs): each thread takes one node and
// a strided share of the element list; partial sums meet in shared memory.
template <typename R>
__global__ void __launch_bounds__(256) k_bnd_near(Geo g, int64_t nbnear, int nrhs, const int32_t *__restrict__ leaf,
                                                  const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                                                  const double *__restrict__ q, R *__restrict__ phib) {
  __shared__ R red[256];
  const int slot = blockIdx.x, rhs = blockIdx.y;
  const int n = g.n, m = g.m, L = g.L, mm = m * m;
  const int ngrp = blockDim.x / mm;
  const int t = threadIdx.x % mm, grp = threadIdx.x / mm;
  int a, b;
  morton_decode((uint32_t)leaf[slot], a, b);
  const R ell = (R)((n + 1.0) / n), invn = R(1) / (R)n, hR = (R)g.h;
  const double *qr = q + (int64_t)rhs * g.NG;
  const int x = a * m + t % m + 1, y = b * m + t / m + 1;
  const int f0 = first[slot], cnt = (first[slot + 1] - f0) * m;
  R acc = 0;
  if (grp < ngrp)
    for (int idx = grp; idx < cnt; idx += ngrp) {
      const int bl = src[f0 + idx / m], e = idx % m;
      const int side = bl >> L;
      const int64_t kk = bl & ((int64_t(1) << L) - 1);
      int u, d;
      side_coords(side, n + 1, x, y, u, d);
      // s1 = t_a - u with t_a = (k m + e)(n + 1)/n: exact integer numerator over n
      const int64_t num = (kk * m + e) * (int64_t)(n + 1) - (int64_t)u * n;
      acc += (R)qr[side * n + kk * m + e] * hR * seg_log_int<R>((R)num * invn, ell, (R)d);
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < mm) {
    R s = 0;
    for (int q2 = 0; q2 < ngrp; ++q2) s += red[q2 * mm + threadIdx.x];
    phib[((int64_t)rhs * nbnear + slot) * mm + threadIdx.x] = s;
  }
}

// Double layer near the boundary: phib[slot][t] (+)= dsgn sum_e dens_e theta_e(x_t), theta_e =
// int_e d/dn_y ln|x - y| ds = -atan2(l d, d^2 + s1 s2) (the signed angle element e subtends at
// the node, outward normal; node units, so no factor h).  Same blocks and element lists as
// k_bnd_near.  accumulate = 0 writes instead of adding (no single layer in that apply).
template <typename R>
__global__ void __launch_bounds__(256) k_dl_near(Geo g, int64_t nbnear, int nrhs, const int32_t *__restrict__ leaf,
                                                 const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                                                 const double *__restrict__ dens, R dsgn, int accumulate,
                                                 R *__restrict__ phib) {
  __shared__ R red[256];
  const int slot = blockIdx.x, rhs = blockIdx.y;
  const int n = g.n, m = g.m, L = g.L, mm = m * m;
  const int ngrp = blockDim.x / mm;
  const int t = threadIdx.x % mm, grp = threadIdx.x / mm;
  int a, b;
  morton_decode((uint32_t)leaf[slot], a, b);
  const R ell = (R)((n + 1.0) / n), invn = R(1) / (R)n;
  const double *dr = dens + (int64_t)rhs * g.NG;
  const int x = a * m + t % m + 1, y = b * m + t / m + 1;
  const int f0 = first[slot], cnt = (first[slot + 1] - f0) * m;
  R acc = 0;
  if (grp < ngrp)
    for (int idx = grp; idx < cnt; idx += ngrp) {
      const int bl = src[f0 + idx / m], e = idx % m;
      const int side = bl >> L;
      const int64_t kk = bl & ((int64_t(1) << L) - 1);
      int u, d;
      side_coords(side, n + 1, x, y, u, d);
      const int64_t num = (kk * m + e) * (int64_t)(n + 1) - (int64_t)u * n;
      const R s1 = (R)num * invn, s2 = s1 + ell, dd = (R)d;
      acc += (R)dr[side * n + kk * m + e] * -atan2(ell * dd, dd * dd + s1 * s2);
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < mm) {
    R sacc = 0;
    for (int q2 = 0; q2 < ngrp; ++q2) sacc += red[q2 * mm + threadIdx.x];
    R *o = phib + ((int64_t)rhs * nbnear + slot) * mm + threadIdx.x;
    *o = (accumulate ? *o : R(0)) + dsgn * sacc;
  }
}

// Point sources at the collocation points next to the boundary (the transpose pass):
// phib[slot][t] = sum_e c_e h^2 ln|x_t - y_e| (node units) over the elements of the leaf's
// near boundary runs; y_e the element midpoint.  Same blocks and lists as k_bnd_near.
template <typename R>
__global__ void __launch_bounds__(256) k_pt_near(Geo g, int64_t nbnear, int nrhs, const int32_t *__restrict__ leaf,
                                                 const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                                                 const double *__restrict__ c, R *__restrict__ phib) {
  __shared__ double red[256];
  const int slot = blockIdx.x, rhs = blockIdx.y;
  const int n = g.n, m = g.m, L = g.L, mm = m * m;
  const int ngrp = blockDim.x / mm;
  const int t = threadIdx.x % mm, grp = threadIdx.x / mm;
  int a, b;
  morton_decode((uint32_t)leaf[slot], a, b);
  const double h2 = g.h * g.h;
  const double *cr = c + (int64_t)rhs * g.NG;
  const int x = a * m + t % m + 1, y = b * m + t / m + 1;
  const int f0 = first[slot], cnt = (first[slot + 1] - f0) * m;
  double acc = 0;
  if (grp < ngrp)
    for (int idx = grp; idx < cnt; idx += ngrp) {
      const int bl = src[f0 + idx / m], e = idx % m;
      const int side = bl >> L;
      const int64_t kk = bl & ((int64_t(1) << L) - 1);
      int u, d;
      side_coords(side, n + 1, x, y, u, d);
      // midpoint minus node along the side: ((2(k m + e) + 1)(n + 1) - 2 u n) / (2n)
      const double ds = (double)((2 * (kk * m + e) + 1) * (int64_t)(n + 1) - 2 * (int64_t)u * n) / (2.0 * n);
      acc += cr[side * n + kk * m + e] * h2 * 0.5 * log(ds * ds + (double)d * (double)d);
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < mm) {
    double sacc = 0;
    for (int q2 = 0; q2 < ngrp; ++q2) sacc += red[q2 * mm + threadIdx.x];
    phib[((int64_t)rhs * nbnear + slot) * mm + threadIdx.x] = (R)sacc;
  }
}

// The transpose pass's boundary values: t_k = int_{element k} Phi(y) dGamma_y / h^2 for the
// volume potential Phi of the weights (h^2 zb) whose local expansions Lb and near nodes the
// collocation pass uses, i.e. (S_OG^T zb)_k = sum_i zb_i int_k G(x_i, y) dGamma.  Far part:
// int_e Re sum_k Lt_k z^k over the element, z the offset from each ancestor run's centre in
// run units, in closed form; near part: the closed-form element integrals of ln|y - x_j|.
// Block per (boundary leaf run, rhs); FP64 arithmetic.
template <typename R>
__global__ void __launch_bounds__(256) k_colloc_T(Geo g, int nrhs, const R *__restrict__ wpad,
                                                  const cpx<R> *__restrict__ Lb, const int32_t *__restrict__ pfirst,
                                                  const int32_t *__restrict__ psrc, double *__restrict__ tout) {
  __shared__ double red[8][16];
  const int n = g.n, m = g.m, L = g.L, p = g.p, mm = m * m;
  const int64_t bl = blockIdx.x;
  const int rhs = blockIdx.y;
  const int side = (int)(bl >> L);
  const int64_t kk = bl & ((int64_t(1) << L) - 1);
  const R *W = wpad + (int64_t)rhs * g.npad * g.npad;
  const double ell = (n + 1.0) / n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int c_near = pfirst[bl + 1] - pfirst[bl];
  for (int e = 0; e < m; ++e) {
    double acc = 0.0;
    for (int it = threadIdx.x; it < c_near * mm; it += blockDim.x) {
      const int el = it / mm, t = it % mm;
      int a, b;
      morton_decode((uint32_t)psrc[pfirst[bl] + el], a, b);
      const int i = a * m + t % m, j = b * m + t / m;
      int u, d;
      side_coords(side, n + 1, i + 1, j + 1, u, d);
      const int64_t num = (kk * m + e) * (int64_t)(n + 1) - (int64_t)u * n;
      acc += (double)W[(int64_t)(j + g.pad) * g.npad + i + g.pad] * seg_log_int<double>((double)num / n, ell, (double)d);
    }
    acc = warp_sum(acc);
    if (lane == 0) red[wid][e] = acc;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    const int e = threadIdx.x;
    double near = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) near += red[w][e];
    const int along = (int)(kk * m + e);  // element index along the side
    const double ex = (side == 0) ? 1.0 : (side == 2 ? -1.0 : 0.0);
    const double ey = (side == 1) ? 1.0 : (side == 3 ? -1.0 : 0.0);
    double far = 0.0;
    for (int l = 0; l <= L; ++l) {
      const int nl = n >> l;
      const int64_t id = ((int64_t)side << l) + along / nl;
      const double o1 = ell * ((double)(along % nl) - 0.5 * nl) / nl, o2 = o1 + ell / nl;
      const cpx<R> *Lc = Lb + (int64_t)rhs * g.nbcell * p + (blevel_offset(l) + id) * p;
      // sum_k Lt_k e^k nl (o2^{k+1} - o1^{k+1}) / (k + 1)
      double pr = 1.0, pi = 0.0, p1 = o1, p2 = o2;  // e^k; o^{k+1}
      for (int k = 0; k < p; ++k) {
        const double w = nl * (p2 - p1) / (k + 1);
        far += w * ((double)Lc[k].re * pr - (double)Lc[k].im * pi);
        const double nr = pr * ex - pi * ey, ni = pr * ey + pi * ex;
        pr = nr;
        pi = ni;
        p1 *= o1;
        p2 *= o2;
      }
    }
    tout[(int64_t)rhs * g.NG + side * n + along] = (near + far) * NEG_INV_2PI / (g.h * g.h) * g.h;
  }
}

// The same integrals formed once at set-up (FP64, stored FP32) for the single-precision
// forms: K[(first[slot] m + idx) m^2 + t] = h int_{element idx} ln|x_t - y| ds, so each apply
// is a product with q instead of ~5e6 log/atan2 evaluations at 1024^2.
__global__ void __launch_bounds__(256) k_bnd_near_mat(Geo g, int64_t nbnear, const int32_t *__restrict__ leaf,
                                                      const int32_t *__restrict__ first,
                                                      const int32_t *__restrict__ src, float *__restrict__ K) {
  const int slot = blockIdx.x;
  const int n = g.n, m = g.m, L = g.L, mm = m * m;
  const int ngrp = blockDim.x / mm;
  const int t = threadIdx.x % mm, grp = threadIdx.x / mm;
  if (grp >= ngrp) return;
  int a, b;
  morton_decode((uint32_t)leaf[slot], a, b);
  const double ell = (n + 1.0) / n;
  const int x = a * m + t % m + 1, y = b * m + t / m + 1;
  const int f0 = first[slot], cnt = (first[slot + 1] - f0) * m;
  for (int idx = grp; idx < cnt; idx += ngrp) {
    const int bl = src[f0 + idx / m], e = idx % m;
    const int side = bl >> L;
    const int64_t kk = bl & ((int64_t(1) << L) - 1);
    int u, d;
    side_coords(side, n + 1, x, y, u, d);
    const int64_t num = (kk * m + e) * (int64_t)(n + 1) - (int64_t)u * n;
    K[((int64_t)f0 * m + idx) * mm + t] = (float)(g.h * seg_log_int<double>((double)num / n, ell, (double)d));
  }
}

// Apply of the precomputed integrals: block per (slot, rhs), 16 groups of 16 threads; a
// thread takes 4 consecutive nodes (float4) of every 16th element; partials meet in shared
// memory.  Requires m = 8 (64 nodes per leaf).
__global__ void __launch_bounds__(256) k_bnd_near_k(Geo g, int64_t nbnear, int nrhs, const int32_t *__restrict__ first,
                                                    const int32_t *__restrict__ src, const float *__restrict__ K,
                                                    const double *__restrict__ q, float *__restrict__ phib) {
  __shared__ float4 red[16][16];
  const int slot = blockIdx.x, rhs = blockIdx.y;
  const int n = g.n, m = g.m, L = g.L;
  const int t4 = threadIdx.x & 15, grp = threadIdx.x >> 4;
  const double *qr = q + (int64_t)rhs * g.NG;
  const int f0 = first[slot], cnt = (first[slot + 1] - f0) * m;
  const float4 *K4 = reinterpret_cast<const float4 *>(K) + (int64_t)f0 * m * 16;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int idx = grp; idx < cnt; idx += 16) {
    const int bl = src[f0 + idx / m], e = idx % m;
    const int64_t kk = bl & ((int64_t(1) << L) - 1);
    const float qe = (float)qr[(bl >> L) * n + kk * m + e];
    const float4 kv = K4[(int64_t)idx * 16 + t4];
    acc.x = fmaf(kv.x, qe, acc.x);
    acc.y = fmaf(kv.y, qe, acc.y);
    acc.z = fmaf(kv.z, qe, acc.z);
    acc.w = fmaf(kv.w, qe, acc.w);
  }
  red[grp][t4] = acc;
  __syncthreads();
  if (threadIdx.x < 64) {
    const int tt = threadIdx.x >> 2, c = threadIdx.x & 3;
    float sacc = 0.f;
    for (int q2 = 0; q2 < 16; ++q2) {
      const float4 v = red[q2][tt];
      sacc += c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
    }
    phib[((int64_t)rhs * nbnear + slot) * 64 + threadIdx.x] = sacc;
  }
}

// ------------------------------------------------------------------ near field (P2P)
// One CTA per tile of TX x TY leaves, one thread per (leaf, row of m targets).  The
// weight image of the tile and its halo of R leaves, and the table of ln|d| over the
// stencil's node offsets (rows |dy| only: the table is even in dy), are staged in shared
// memory.  For every stencil row oy and source row sy a thread slides along the
// contiguous run of source leaves: per source leaf it loads the m weights of the row and
// the 2m-1 table values of the window and does m x m FMAs.  The sum over a stencil row is
// folded into Kahan-compensated accumulators (Sec. 7.1).  out = -near / (2 pi).
template <typename R>
struct P2PArgs {
  const R *wpad;
  const R *table;
  double *out;
  int n, npad, L, R_, Rn, HX, HY, TS, c0, tile_x, tile_y, nrhs;
  Stencil st;
};

template <typename R, int K>
__device__ __forceinline__ void lds_vec(const R *__restrict__ p, R (&v)[K]) {
  constexpr int VW = 16 / sizeof(R);
  static_assert(K % VW == 0, "vector width");
#pragma unroll
  for (int i = 0; i < K; i += VW) {
    if constexpr (sizeof(R) == 4) {
      float4 t = *reinterpret_cast<const float4 *>(p + i);
      v[i] = t.x; v[i + 1] = t.y; v[i + 2] = t.z; v[i + 3] = t.w;
    } else {
      double2 t = *reinterpret_cast<const double2 *>(p + i);
      v[i] = t.x; v[i + 1] = t.y;
    }
  }
}

template <typename R, int M>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_p2p(P2PArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *halo = reinterpret_cast<R *>(smem_raw);
  R *tab = halo + (int64_t)A.HY * A.HX;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rhs = blockIdx.z;
  const int lx0 = blockIdx.x * A.tile_x, ly0 = blockIdx.y * A.tile_y;
  {
    const R *W = A.wpad + (int64_t)rhs * A.npad * A.npad;
    constexpr int VW = 16 / sizeof(R);
    const int vx = A.HX / VW;
    for (int idx = tid; idx < A.HY * vx; idx += nthr) {
      const int r = idx / vx, cv = idx - r * vx;
      const R *src = W + (int64_t)(ly0 * M + r) * A.npad + lx0 * M + cv * VW;
      R *dst = halo + r * A.HX + cv * VW;
      if constexpr (sizeof(R) == 4)
        *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(src);
      else
        *reinterpret_cast<double2 *>(dst) = *reinterpret_cast<const double2 *>(src);
    }
    const int tv = (A.Rn + 1) * A.TS / VW;
    for (int idx = tid; idx < tv; idx += nthr) {
      if constexpr (sizeof(R) == 4)
        reinterpret_cast<float4 *>(tab)[idx] = reinterpret_cast<const float4 *>(A.table)[idx];
      else
        reinterpret_cast<double2 *>(tab)[idx] = reinterpret_cast<const double2 *>(A.table)[idx];
    }
  }
  __syncthreads();
  const int ty = tid % M, li = tid / M;
  const int lxl = li % A.tile_x, lyl = li / A.tile_x;
  R sum[M], comp[M];
#pragma unroll
  for (int t = 0; t < M; ++t) sum[t] = comp[t] = 0;
  const int Rr = A.R_;
  for (int oy = -Rr; oy <= Rr; ++oy) {
    const int ox0 = A.st.ox0[oy + Rr], ox1 = A.st.ox1[oy + Rr];
    if (ox0 > ox1) continue;
    R part[M];
#pragma unroll
    for (int t = 0; t < M; ++t) part[t] = 0;
    for (int sy = 0; sy < M; ++sy) {
      const R *hrow = halo + ((lyl + Rr + oy) * M + sy) * A.HX + (lxl + Rr) * M;
      const int dy = -oy * M + ty - sy;
      const R *trow = tab + (dy < 0 ? -dy : dy) * A.TS + A.c0 + A.Rn - (M - 1);
      for (int c = ox0; c <= ox1; ++c) {
        R w[M], tw[2 * M];
        lds_vec<R, M>(hrow + c * M, w);
        lds_vec<R, 2 * M>(trow - c * M, tw);
#pragma unroll
        for (int tx = 0; tx < M; ++tx)
#pragma unroll
          for (int sx = 0; sx < M; ++sx) part[tx] = fma(w[sx], tw[tx - sx + M - 1], part[tx]);
      }
    }
#pragma unroll
    for (int t = 0; t < M; ++t) {  // Kahan
      const R y = part[t] - comp[t];
      const R s = sum[t] + y;
      comp[t] = (s - sum[t]) - y;
      sum[t] = s;
    }
  }
  const int gx = lx0 + lxl, gy = ly0 + lyl;
  double *o = A.out + (int64_t)rhs * A.n * A.n + (int64_t)(gy * M + ty) * A.n + gx * M;
#pragma unroll
  for (int t = 0; t < M; ++t) o[t] = ((double)sum[t] - (double)comp[t]) * NEG_INV_2PI;
}

// -(1/2pi) (a + b) + u, u = v (float)(-1/2pi): a + b exactly as a two-word sum (Knuth's
// TwoSum), times -1/(2pi) held as two floats (the product's error word from an FMA, as in
// Dekker's product), u added with TwoSum, and the two words converted to FP64 and added.
__device__ __forceinline__ double near_far_sum(float a, float b, float v) {
  constexpr float c_hi = (float)NEG_INV_2PI;
  constexpr float c_lo = (float)(NEG_INV_2PI - (double)c_hi);
  const float s = a + b, bb = s - a, s_lo = (a - (s - bb)) + (b - bb);
  const float p = __fmul_rn(s, c_hi);  // rounded products, never fused into the sums below
  const float p_lo = fmaf(s, c_hi, -p) + fmaf(s, c_lo, s_lo * c_hi);
  const float u = __fmul_rn(v, c_hi);
  const float r = p + u, rb = r - p, r_lo = ((p - (r - rb)) + (u - rb)) + p_lo;
  return f32_to_f64_bits(r) + f32_to_f64_bits(r_lo);
}

// The whole downward pass of the volume tree, L2L (item 4) and L2P (item 5), in one launch,
// with the final sum z = -(1/2pi) (near field + far field + near-boundary correction).
// Block (b, rhs) takes the 4x4 Morton block b of leaves (cell b of level L - 2): it first
// forms the complete local expansion of each of its ancestors from the root down (its own
// copy: L(cell) = L_M2L(cell) + L2L(L(parent)), at most P terms per output), then those of
// cell b, its 4 children and the 16 leaves, and evaluates each leaf expansion at the leaf's
// nodes (NPT consecutive nodes of one row per thread, so a warp writes whole row segments).
template <typename R, int P, int M>
__global__ void __launch_bounds__(256) k_downward_tree(Geo g, int nrhs, int do_bnd, int64_t nbnear,
                                                       const cpx<R> *__restrict__ Mv, const cpx<R> *__restrict__ Mb,
                                                       int with_bnd_w, const cpx<R> *__restrict__ vl2l,
                                                       const cpx<R> *__restrict__ Lv, const int32_t *__restrict__ vslot,
                                                       const cpx<R> *__restrict__ Lsep, int64_t nsep,
                                                       const R *__restrict__ phib, const int32_t *__restrict__ bslot,
                                                       double *__restrict__ out, const float *__restrict__ near1,
                                                       const float *__restrict__ near2) {
  __shared__ cpx<R> sS[4 * P * P], sanc[24][P], s1[4][P], s2[16][P];
  const int tid = threadIdx.x, nthr = blockDim.x, rhs = blockIdx.y;
  const uint32_t blk = blockIdx.x;
  const int L = g.L;
  const cpx<R> *Lr = Lv + (int64_t)rhs * g.ncell * P;

  // every value the block needs, loaded at once: the translation matrices, the M2L parts of
  // the ancestors (levels 0 .. L - 2), of the 4 children and of the 16 leaves
  for (int i = tid; i < 4 * P * P; i += nthr) sS[i] = vl2l[i];
  // L of cell c (global index), coefficient n, with the boundary-source part kept apart
  auto lval = [&](int64_t c, int n) -> cpx<R> {
    cpx<R> v = Lr[c * P + n];
    if (vslot) {
      const int sl = vslot[c];
      if (sl >= 0) v = v + Lsep[((int64_t)rhs * nsep + sl) * P + n];
    }
    return v;
  };
  for (int i = tid; i < (L - 1) * P; i += nthr) {
    const int l = i / P, n = i % P;
    sanc[l][n] = lval(level_offset(l) + (blk >> (2 * (L - 2 - l))), n);
  }
  for (int i = tid; i < 4 * P; i += nthr) s1[i / P][i % P] = lval(level_offset(L - 1) + 4 * blk + i / P, i % P);
  for (int i = tid; i < 16 * P; i += nthr) s2[i / P][i % P] = lval(level_offset(L) + 16 * blk + i / P, i % P);
  if (tid == 0) {  // the root also takes ln h times the total weight (volume, and boundary if present)
    double W = (double)Mv[(int64_t)rhs * g.ncell * P].re;
    if (with_bnd_w)
      for (int sd = 0; sd < 4; ++sd) W += (double)Mb[((int64_t)rhs * g.nbcell + sd) * P].re;
    sanc[0][0].re = sanc[0][0].re + (R)(g.lnh * W);
  }
  __syncthreads();
  // complete local expansions down the ancestor chain, in place: sanc[l] += L2L(sanc[l - 1]),
  // by the first warp alone (P <= 32 outputs per step), so the steps meet at warp barriers
  // and the other warps wait at a single block barrier
  if (tid < 32) {
    for (int l = 1; l <= L - 2; ++l) {
      const int q = (blk >> (2 * (L - 2 - l))) & 3;
      cpx<R> acc = mk<R>(0, 0);
      if (tid < P) {
        const int n = tid;
        acc = sanc[l][n];
#pragma unroll
        for (int k = 0; k < P; ++k)
          if (k >= n) cmac(acc, sS[(q * P + n) * P + k], sanc[l - 1][k]);
      }
      __syncwarp();
      if (tid < P) sanc[l][tid] = acc;
      __syncwarp();
    }
  }
  __syncthreads();
  const cpx<R> *cur = sanc[L - 2];
  cpx<R> v1 = mk<R>(0, 0), v2 = mk<R>(0, 0);
  if (tid < 4 * P) {
    const int q = tid / P, n = tid % P;
    v1 = s1[q][n];
#pragma unroll
    for (int k = 0; k < P; ++k)
      if (k >= n) cmac(v1, sS[(q * P + n) * P + k], cur[k]);
  }
  __syncthreads();
  if (tid < 4 * P) s1[tid / P][tid % P] = v1;
  __syncthreads();
  if (tid < 16 * P) {
    const int lf = tid / P, n = tid % P, q = lf & 3;
    v2 = s2[lf][n];
#pragma unroll
    for (int k = 0; k < P; ++k)
      if (k >= n) cmac(v2, sS[(q * P + n) * P + k], s1[lf >> 2][k]);
  }
  __syncthreads();
  if (tid < 16 * P) s2[tid / P][tid % P] = v2;
  __syncthreads();
  constexpr int NPT = M * M / 16;  // nodes per thread: (4M)^2 nodes over 256 threads
  const int e0 = tid * NPT, y = e0 / (4 * M), x0 = e0 % (4 * M);
  const int lf = (int)morton_encode((uint32_t)(x0 / M), (uint32_t)(y / M));
  const int tx0 = x0 % M, ty = y % M;
  int bx, by;
  morton_decode(blk, bx, by);
  const int64_t off = (int64_t)rhs * g.n * g.n + (int64_t)(by * 4 * M + y) * g.n + bx * 4 * M + x0;
  const R *pb = nullptr;
  if (do_bnd) {
    const int slot = bslot[16 * (int64_t)blk + lf];
    if (slot >= 0) pb = phib + ((int64_t)rhs * nbnear + slot) * M * M + ty * M + tx0;
  }
  const R zy = (ty - R(0.5) * (M - 1)) / M;
  cpx<R> acc[NPT];
#pragma unroll
  for (int e = 0; e < NPT; ++e) acc[e] = mk<R>(0, 0);
  for (int k = P - 1; k >= 0; --k) {
    const cpx<R> Lk = s2[lf][k];
#pragma unroll
    for (int e = 0; e < NPT; ++e) acc[e] = acc[e] * mk<R>((tx0 + e - R(0.5) * (M - 1)) / M, zy) + Lk;
  }
  double *o = out + off;
  if (near1) {
    // tensor-core near field: the two raw halves often cancel, so they are added exactly
    // and scaled by -1/(2 pi) in two-word FP32 arithmetic, the far term added, and the
    // two-word result converted to FP64 with one FP64 addition (FP64 is scarce here)
#pragma unroll
    for (int e = 0; e < NPT; ++e) {
      float v = (float)acc[e].re;
      if (pb) v += (float)pb[e];
      o[e] = near_far_sum(near1[off + e], near2[off + e], v);
    }
  } else {
#pragma unroll
    for (int e = 0; e < NPT; ++e) {
      double v = (double)acc[e].re;
      if (pb) v += (double)pb[e];
      o[e] += v * NEG_INV_2PI;
    }
  }
}

// z += -(1/2pi) (L2P of the leaf local expansion + near-boundary element integrals).
// Thread per (leaf, row of m targets, rhs).
template <typename R, int M>
__global__ void k_far_final(int n, int L, int p, int64_t ncell, int64_t nbnear, int nrhs, int do_bnd,
                            const cpx<R> *__restrict__ Lv, const R *__restrict__ phib,
                            const int32_t *__restrict__ bslot, double *__restrict__ out,
                            const float *__restrict__ near1, const float *__restrict__ near2) {
  const int64_t nleaf = int64_t(1) << (2 * L);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nleaf * M * nrhs) return;
  const int ty = (int)(t % M);
  const int64_t rest = t / M, leafc = rest % nleaf;
  const int rhs = (int)(rest / nleaf);
  int gx, gy;
  morton_decode((uint32_t)leafc, gx, gy);
  const cpx<R> *Lc = Lv + (int64_t)rhs * ncell * p + (level_offset(L) + leafc) * p;
  const R zy = (ty - R(0.5) * (M - 1)) / M;
  cpx<R> acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = mk<R>(0, 0);
  for (int k = p - 1; k >= 0; --k) {
    const cpx<R> Lk = Lc[k];
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] = acc[q] * mk<R>((q - R(0.5) * (M - 1)) / M, zy) + Lk;
  }
  const R *pb = nullptr;
  if (do_bnd) {
    const int slot = bslot[leafc];
    if (slot >= 0) pb = phib + ((int64_t)rhs * nbnear + slot) * M * M + ty * M;
  }
  const int64_t off = (int64_t)rhs * n * n + (int64_t)(gy * M + ty) * n + gx * M;
  double *o = out + off;
  if (near1) {
    // tensor-core near field: the two raw halves and the far term meet in FP64 (they often
    // cancel) -- one add and one fused multiply-add per node
#pragma unroll
    for (int q = 0; q < M; ++q) {
      float v = (float)acc[q].re;
      if (pb) v += (float)pb[q];
      o[q] = fma((double)near1[off + q] + (double)near2[off + q], NEG_INV_2PI, (double)(v * (float)NEG_INV_2PI));
    }
  } else {
#pragma unroll
    for (int q = 0; q < M; ++q) {
      double v = (double)acc[q].re;
      if (pb) v += (double)pb[q];
      o[q] += v * NEG_INV_2PI;
    }
  }
}

// P2M for trees with L < 2 (n <= 2 m): warp per leaf in one block.
template <typename R, int P>
__global__ void k_p2m_small(Geo g, int nrhs, const R *__restrict__ wpad, cpx<R> *__restrict__ Mv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nw = g.nleaf * nrhs;
  for (int64_t wi = w; wi < nw; wi += blockDim.x / 32) {
    const int rhs = (int)(wi / g.nleaf);
    const uint32_t c = (uint32_t)(wi % g.nleaf);
    cpx<R> acc[P];
    p2m_warp<R, P>(wpad + (int64_t)rhs * g.npad * g.npad, g.npad, g.pad, g.m, c, lane, acc);
    if (lane == 0)
      for (int k = 0; k < P; ++k) Mv[(int64_t)rhs * g.ncell * P + (level_offset(g.L) + c) * P + k] = acc[k];
  }
}

// ------------------------------------------------------------------ host side
template <typename R, int M>
size_t p2p_smem(const P2PArgs<R> &a) {
  return ((size_t)a.HY * a.HX + (size_t)(a.Rn + 1) * a.TS) * sizeof(R);
}

template <typename R, int M>
void launch_p2p(int L, const P2PArgs<R> &a, cudaStream_t s) {
  const int side = 1 << L;
  dim3 grid(side / a.tile_x, side / a.tile_y, a.nrhs);
  const int threads = a.tile_x * a.tile_y * M;
  k_p2p<R, M><<<grid, threads, p2p_smem<R, M>(a), s>>>(a);
  FMMPC_LAUNCH_CHECK();
}

// Kernels that need more than 48 KB of dynamic shared memory: raise their limit once, at
// set-up (the attribute is per function), to the per-block maximum minus static use.
template <typename K>
void raise_smem_limit(K kernel) {
  cudaFuncAttributes fa{};
  FMMPC_CUDA(cudaFuncGetAttributes(&fa, kernel));
  int dev = 0, optin = 0;
  FMMPC_CUDA(cudaGetDevice(&dev));
  FMMPC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  FMMPC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
}

template <typename R>
void set_p2p_smem_limit() {
  raise_smem_limit(k_p2p<R, 4>);
  raise_smem_limit(k_p2p<R, 8>);
  raise_smem_limit(k_p2p<R, 16>);
}

template <typename R>
void run_p2p(fmmpc_handle &H, const void *table, double *out, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  P2PArgs<R> a{};
  a.wpad = (const R *)H.fb.wpad;
  a.table = (const R *)table;
  a.out = out;
  a.n = g.n; a.npad = g.npad; a.L = g.L; a.R_ = g.R; a.Rn = H.fb.Rn;
  a.HX = (H.tile_x + 2 * g.R) * g.m;
  a.HY = (H.tile_y + 2 * g.R) * g.m;
  a.TS = H.fb.table_stride; a.c0 = H.fb.table_c0;
  a.tile_x = H.tile_x; a.tile_y = H.tile_y; a.nrhs = nrhs;
  a.st = H.st;
  switch (g.m) {
    case 4: launch_p2p<R, 4>(g.L, a, s); break;
    case 8: launch_p2p<R, 8>(g.L, a, s); break;
    case 16: launch_p2p<R, 16>(g.L, a, s); break;
    default: throw Error(FMMPC_ERR_UNSUPPORTED, "leaf side must be 4, 8 or 16");
  }
}

template <typename R>
void run_far_final(fmmpc_handle &H, double *out, int nrhs, int do_bnd, cudaStream_t s,
                   const float *near1 = nullptr, const float *near2 = nullptr) {
  const Geo &g = H.g;
  const int64_t tasks = g.nleaf * g.m * nrhs;
  const cpx<R> *Lv = (const cpx<R> *)H.fb.Lv;
  const R *pb = (const R *)H.fb.phib;
  switch (g.m) {
    case 4: k_far_final<R, 4><<<nblk(tasks, 128), 128, 0, s>>>(g.n, g.L, g.p, g.ncell, H.lists.nbnear, nrhs, do_bnd, Lv, pb, H.lists.leaf_bslot, out, near1, near2); break;
    case 8: k_far_final<R, 8><<<nblk(tasks, 128), 128, 0, s>>>(g.n, g.L, g.p, g.ncell, H.lists.nbnear, nrhs, do_bnd, Lv, pb, H.lists.leaf_bslot, out, near1, near2); break;
    default: k_far_final<R, 16><<<nblk(tasks, 128), 128, 0, s>>>(g.n, g.L, g.p, g.ncell, H.lists.nbnear, nrhs, do_bnd, Lv, pb, H.lists.leaf_bslot, out, near1, near2); break;
  }
  FMMPC_LAUNCH_CHECK();
}

template <typename R>
Mats<R> mats_of(fmmpc_handle &H) {
  const int P = H.g.p;
  const cpx<R> *base = (const cpx<R> *)H.fb.mats;
  Mats<R> mt;
  mt.vm2m = base;
  mt.vl2l = base + 4 * P * P;
  // each kind holds sum over l = 0..L of 4 (n >> l) P entries = 4 P (2n - m)
  const int64_t lvsize = (int64_t)4 * P * (2 * H.g.n - H.g.m);
  mt.lvq = base + 8 * P * P;
  mt.lvd = mt.lvq + lvsize;
  mt.lvp = mt.lvd + lvsize;
  return mt;
}

// Upward pass of the volume tree: one launch for L >= 2 (P2M, then every M2M level).
template <typename R, int P>
int run_upward(fmmpc_handle &H, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  const R *wpad = (const R *)H.fb.wpad;
  cpx<R> *Mv = (cpx<R> *)H.fb.Mv;
  Mats<R> mt = mats_of<R>(H);
  if (g.L >= 2) {
    const dim3 grid((unsigned)(int64_t(1) << (2 * (g.L - 2))), nrhs);
    switch (g.m) {
      case 4: k_upward_tree<R, P, 4><<<grid, 256, 0, s>>>(g, wpad, mt.vm2m, Mv, H.fb.up_count, H.fb.up_ncount); break;
      case 8: k_upward_tree<R, P, 8><<<grid, 256, 0, s>>>(g, wpad, mt.vm2m, Mv, H.fb.up_count, H.fb.up_ncount); break;
      case 16: k_upward_tree<R, P, 16><<<grid, 256, 0, s>>>(g, wpad, mt.vm2m, Mv, H.fb.up_count, H.fb.up_ncount); break;
      default: throw Error(FMMPC_ERR_UNSUPPORTED, "leaf side must be 4, 8 or 16");
    }
    FMMPC_LAUNCH_CHECK();
    return 1;
  }
  k_p2m_small<R, P><<<1, 256, 0, s>>>(g, nrhs, wpad, Mv);
  if (g.L == 1) k_m2m_levels<R, P><<<1, 256, 0, s>>>(0, 0, g.ncell, nrhs, mt.vm2m, Mv);
  FMMPC_LAUNCH_CHECK();
  return g.L == 1 ? 2 : 1;
}

// Downward pass for trees of depth L < 2 (one launch per level; deeper trees use the
// one-launch downward kernel).
template <typename R, int P>
int run_l2l(fmmpc_handle &H, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  cpx<R> *Lv = (cpx<R> *)H.fb.Lv;
  Mats<R> mt = mats_of<R>(H);
  int launches = 0;
  for (int lp = 0; lp < g.L; ++lp) {
    const int64_t tasks = (int64_t(1) << (2 * (lp + 1))) * P * nrhs;
    k_l2l_levels<R, P><<<nblk(tasks), 256, 0, s>>>(lp, lp + 1, g.ncell, nrhs, mt.vl2l, Lv);
    ++launches;
  }
  FMMPC_LAUNCH_CHECK();
  return launches;
}

// L2L and L2P with the final sum in one launch (L >= 2); with_bnd_w: the root constant
// includes the boundary weight.
template <typename R, int P>
void run_downward(fmmpc_handle &H, double *out, int nrhs, int do_bnd, int with_bnd_w, cudaStream_t s,
                  const float *near1 = nullptr, const float *near2 = nullptr, bool sep = false) {
  const Geo &g = H.g;
  const int32_t *vslot = sep ? H.lists.vbv_slot : nullptr;
  const cpx<R> *Lsep = (const cpx<R> *)H.fb.Lvb;
  const int64_t nsep = H.lists.n_vbv_cells;
  const cpx<R> *Mv = (const cpx<R> *)H.fb.Mv, *Mb = (const cpx<R> *)H.fb.Mb;
  const cpx<R> *Lv = (const cpx<R> *)H.fb.Lv;
  const R *pb = (const R *)H.fb.phib;
  const cpx<R> *vl2l = mats_of<R>(H).vl2l;
  const dim3 grid((unsigned)(int64_t(1) << (2 * (g.L - 2))), nrhs);
  switch (g.m) {
    case 4: k_downward_tree<R, P, 4><<<grid, 256, 0, s>>>(g, nrhs, do_bnd, H.lists.nbnear, Mv, Mb, with_bnd_w, vl2l, Lv, vslot, Lsep, nsep, pb, H.lists.leaf_bslot, out, near1, near2); break;
    case 8: k_downward_tree<R, P, 8><<<grid, 256, 0, s>>>(g, nrhs, do_bnd, H.lists.nbnear, Mv, Mb, with_bnd_w, vl2l, Lv, vslot, Lsep, nsep, pb, H.lists.leaf_bslot, out, near1, near2); break;
    case 16: k_downward_tree<R, P, 16><<<grid, 256, 0, s>>>(g, nrhs, do_bnd, H.lists.nbnear, Mv, Mb, with_bnd_w, vl2l, Lv, vslot, Lsep, nsep, pb, H.lists.leaf_bslot, out, near1, near2); break;
    default: throw Error(FMMPC_ERR_UNSUPPORTED, "leaf side must be 4, 8 or 16");
  }
  FMMPC_LAUNCH_CHECK();
}


// Near-boundary correction phib at the nodes of the leaves next to the boundary.
template <typename R>
int run_bnd_near(fmmpc_handle &H, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  const Lists &Ls = H.lists;
  const dim3 grid((unsigned)Ls.nbnear, nrhs);
  if (H.trans_pass) {  // point sources c' at the collocation points (transpose pass)
    k_pt_near<R><<<grid, 256, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_leaf, Ls.pbv_first, Ls.pbv_src, H.fb.q,
                                      (R *)H.fb.phib);
    FMMPC_LAUNCH_CHECK();
    return 1;
  }
  if (H.bem_form == 1) {  // double-layer correction: D mu only (mu in fb.q)
    k_dl_near<R><<<grid, 256, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_leaf, Ls.pbv_first, Ls.pbv_src, H.fb.q, R(1), 0,
                                      (R *)H.fb.phib);
    FMMPC_LAUNCH_CHECK();
    return 1;
  }
  if (std::is_same<R, float>::value && H.fb.knear && g.m == 8)
    k_bnd_near_k<<<grid, 256, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_first, Ls.pbv_src, H.fb.knear, H.fb.q,
                                      (float *)H.fb.phib);
  else
    k_bnd_near<R><<<grid, 256, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_leaf, Ls.pbv_first, Ls.pbv_src, H.fb.q,
                                       (R *)H.fb.phib);
  FMMPC_LAUNCH_CHECK();
  if (H.bc_g) {  // boundary data: - D g of Eq. e:uinter
    k_dl_near<R><<<grid, 256, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_leaf, Ls.pbv_first, Ls.pbv_src, H.bc_g, R(-1), 1,
                                      (R *)H.fb.phib);
    FMMPC_LAUNCH_CHECK();
    return 2;
  }
  return 1;
}

template <typename R, int P>
void apply_impl(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  const Geo &g = H.g;
  const Lists &Ls = H.lists;
  cudaStream_t s = H.stream;
  GeoDev gd{g.n, g.L, g.tnum, g.tden};
  R *wpad = (R *)H.fb.wpad;
  cpx<R> *Mv = (cpx<R> *)H.fb.Mv, *Lv = (cpx<R> *)H.fb.Lv;
  cpx<R> *Mb = (cpx<R> *)H.fb.Mb, *Lb = (cpx<R> *)H.fb.Lb;
  Mats<R> mt = mats_of<R>(H);
  int64_t launches = 0;
  const int64_t N = (int64_t)g.n * g.n;
  // stage marks: event k opens stage k; a stage that does not run keeps stage_hit = false
  int cur = -1;
  auto mark = [&](int stage) {
    if (!H.timing) return;
    if (H.timing == 2) {  // events only around the M2L (5 -> 6) and P2P (9 -> 10) stages
      if (stage == 5 || stage == 6 || stage == 9 || stage == 10) {
        FMMPC_CUDA(cudaEventRecordWithFlags(H.ev[stage], s, cudaEventRecordExternal));
        H.stage_hit[stage] = true;
      }
      return;
    }
    // external record nodes keep the events timeable when the apply is captured in a graph
    FMMPC_CUDA(cudaEventRecordWithFlags(H.ev[stage], s, cudaEventRecordExternal));
    if (cur >= 0) H.stage_hit[cur] = true;
    cur = stage;
  };
  auto mark_end = [&]() {
    if (!H.timing || H.timing == 2) return;
    FMMPC_CUDA(cudaEventRecordWithFlags(H.ev[fmmpc_handle::NSTAGE], s, cudaEventRecordExternal));
    if (cur >= 0) H.stage_hit[cur] = true;
  };
  if (H.timing)
    for (int k = 0; k < fmmpc_handle::NSTAGE; ++k) H.stage_hit[k] = false;
  mark(0);
  const bool tc = std::is_same<R, float>::value && H.tcp.enabled && H.p2p_engine == 0;
  if (tc) {
    launches += prep_p2p_tc(H, r, nrhs, s, (float *)wpad);  // strips and weight image in one pass
  } else {
    k_weights<R><<<nblk(N * nrhs), 256, 0, s>>>(g.n, g.npad, g.pad, g.h * g.h, N * nrhs, r, wpad);
    FMMPC_LAUNCH_CHECK();
    ++launches;
  }
  if (part == PART_NEAR) {
    mark(9);
    if (tc) {
      launches += run_p2p_tc(H, true, out, nrhs, s);
      launches += add_near2(H, out, nrhs, s);
    }
    else { run_p2p<R>(H, H.fb.table_lnh, out, nrhs, s); ++launches; }
    mark_end();
    H.launches = launches;
    return;
  }
  const bool with_bnd =
      part == PART_FULL || part == PART_VCOL || part == PART_Q || part == PART_BC || part == PART_TRANS;
  const bool trans = part == PART_TRANS;       // P^{-T}: element integrals, S^{-T}, point sources
  const bool dl = H.bem_form == 1;             // double-layer correction (mu from -1/2 I + K)
  const bool bc = part == PART_BC && H.bc_g;   // boundary data g (Eqs. e:ubound / e:uinter)
  // The tensor-core near field and volume M2L do not depend on the boundary chain
  // (collocation values, BEM density, boundary tree, near-boundary correction): for the
  // full apply without stage timing they run on a second stream, forked after the weights
  // and after the upward pass and joined before the boundary-to-volume M2L.
  const bool side = tc && part == PART_FULL && H.timing == 0 && H.sstream;
  const bool m2l_side = side && std::is_same<R, float>::value && H.tcm.enabled;
  cudaStream_t ss = H.sstream;
  // the near part of the collocation values needs only the weights: with the side streams
  // it runs on the third one beside the volume upward pass, and the collocation kernel on
  // the main stream adds the far part
  const bool split_colloc = side && with_bnd && part != PART_TRANS && H.fb.vnear && H.fb.kcol;
  if (side) {
    FMMPC_CUDA(cudaEventRecord(H.sev[0], s));
    FMMPC_CUDA(cudaStreamWaitEvent(ss, H.sev[0], 0));
    launches += run_p2p_tc(H, false, out, nrhs, ss);
    if (split_colloc) {
      FMMPC_CUDA(cudaStreamWaitEvent(H.sstream2, H.sev[0], 0));
      k_colloc<R><<<(unsigned)((int64_t)g.n * nrhs), 128, 0, H.sstream2>>>(
          g, nrhs, wpad, Lb, Ls.pvb_first, Ls.pvb_src, H.fb.vcol, H.fb.kcol, nullptr, nullptr, 1, (R *)H.fb.vnear);
      FMMPC_LAUNCH_CHECK();
      ++launches;
      FMMPC_CUDA(cudaEventRecord(H.sev[6], H.sstream2));
    }
  }
  mark(1);
  launches += run_upward<R, P>(H, nrhs, s);
  if (m2l_side) {  // its own stream, so that it need not wait for the near field
    FMMPC_CUDA(cudaEventRecord(H.sev[1], s));
    FMMPC_CUDA(cudaStreamWaitEvent(H.sstream3, H.sev[1], 0));
    launches += run_m2l_tc(H, Mv, Lv, nrhs, H.sstream3);
    FMMPC_CUDA(cudaEventRecord(H.sev[5], H.sstream3));
  }
  if (with_bnd) {
    mark(2);
    k_m2l_bnd<R, P><<<nblk(g.nbcell * nrhs * 32), 256, 0, s>>>(gd, g.ncell, g.nbcell, nrhs, Ls.vbb_first,
                                                              Ls.vbb_src, Mv, Lb, g.lnh);
    // the side DFT for the two-word BEM apply, fused (not with boundary data, which changes
    // vcol after this kernel)
    const bool vt_f2 = H.Sinv_hi && H.fb.vt_hi && !bc && !trans;
    if (trans)  // t = S_OG^T zb: element integrals of the volume potential, into vcol
      k_colloc_T<R><<<dim3((unsigned)g.nbleaf, nrhs), 256, 0, s>>>(g, nrhs, wpad, Lb, Ls.pvb_first, Ls.pvb_src,
                                                                   H.fb.vcol);
    else {
      if (split_colloc) FMMPC_CUDA(cudaStreamWaitEvent(s, H.sev[6], 0));
      k_colloc<R><<<(unsigned)((int64_t)g.n * nrhs), 128, 0, s>>>(g, nrhs, wpad, Lb, Ls.pvb_first, Ls.pvb_src,
                                                                 H.fb.vcol, H.fb.kcol, vt_f2 ? H.fb.vt_hi : nullptr,
                                                                 vt_f2 ? H.fb.vt_lo : nullptr, split_colloc ? 2 : 0,
                                                                 (R *)H.fb.vnear);
    }
    FMMPC_LAUNCH_CHECK();
    launches += 2;
    if (bc) {  // vcol -= (1/2 I + K) g: Eq. e:ubound's data term
      k_dl_colloc<<<dim3((unsigned)g.NG, nrhs), 256, 0, s>>>(g.n, nrhs, H.bc_g, H.fb.vcol);
      FMMPC_LAUNCH_CHECK();
      ++launches;
    }
    if (part == PART_VCOL) {
      FMMPC_CUDA(cudaMemcpyAsync(out, H.fb.vcol, sizeof(double) * g.NG * nrhs, cudaMemcpyDeviceToDevice, s));
      mark_end();
      H.launches = launches;
      return;
    }
    mark(3);
    // q = S^{-1}(-vcol), or mu = (-1/2 I + K)^{-1}(-vcol) in the double-layer form
    const float *Th = dl ? H.Kdl_hi : H.Sinv_hi, *Tl = dl ? H.Kdl_lo : H.Sinv_lo;
    if (vt_f2 && Th) {  // vt_hi / vt_lo came with the collocation values
      const unsigned nb = (unsigned)((g.n + BEM_ROWS - 1) / BEM_ROWS);
      if (nrhs >= 4) k_bem_apply_f2<4><<<nb, 64 * BEM_ROWS, 0, s>>>(g.n, nrhs, Th, Tl, H.fb.vt_hi, H.fb.vt_lo, H.fb.q);
      else k_bem_apply_f2<1><<<nb, 64 * BEM_ROWS, 0, s>>>(g.n, nrhs, Th, Tl, H.fb.vt_hi, H.fb.vt_lo, H.fb.q);
      ++launches;
    } else {
      k_bem_vt<<<nblk((int64_t)nrhs * g.n), 256, 0, s>>>(g.n, nrhs, H.fb.vcol, H.fb.vt);
      k_bem_apply<<<g.n, 256, 0, s>>>(g.n, nrhs, dl ? H.Kdl_inv : (trans ? H.SinvT : H.Sinv), H.fb.vt, H.fb.q);
      launches += 2;
    }
    FMMPC_LAUNCH_CHECK();
    if (part == PART_Q) {
      FMMPC_CUDA(cudaMemcpyAsync(out, H.fb.q, sizeof(double) * g.NG * nrhs, cudaMemcpyDeviceToDevice, s));
      mark_end();
      H.launches = launches;
      return;
    }
    if (side && Ls.nbnear > 0) {  // the near-boundary correction needs only q: a third stream
      FMMPC_CUDA(cudaEventRecord(H.sev[3], s));
      FMMPC_CUDA(cudaStreamWaitEvent(H.sstream2, H.sev[3], 0));
      launches += run_bnd_near<R>(H, nrhs, H.sstream2);
      FMMPC_CUDA(cudaEventRecord(H.sev[4], H.sstream2));
    }
    mark(4);
    {
      // single layer q (none in the double-layer form); double layer mu (+D mu) or data g
      // (-D g); the transpose pass places point sources h^2 c' at the collocation points
      const double *qm = dl ? nullptr : H.fb.q, *qd = dl ? H.fb.q : (bc ? H.bc_g : nullptr);
      const R dsgn = dl ? R(1) : R(-1);
      const cpx<R> *bq = trans ? mt.lvp : mt.lvq;
      const R qscale = trans ? (R)(g.h * g.h) : (R)g.h;
      const int Lc = H.fb.bup_lc;
      const dim3 grid((unsigned)bup_blocks(g.n, g.L), nrhs);
      cpx<R> *bpart = (cpx<R> *)H.fb.bup_part;
      int *bcnt = H.fb.bup_cnt;
      if (qm && qd)
        k_bnd_up_lv<R, P, true, true><<<grid, 256, 0, s>>>(g, nrhs, Lc, qm, bq, qscale, qd, mt.lvd, dsgn, Mb, bpart, bcnt);
      else if (qm)
        k_bnd_up_lv<R, P, true, false><<<grid, 256, 0, s>>>(g, nrhs, Lc, qm, bq, qscale, qd, mt.lvd, dsgn, Mb, bpart, bcnt);
      else if (qd)
        k_bnd_up_lv<R, P, false, true><<<grid, 256, 0, s>>>(g, nrhs, Lc, qm, bq, qscale, qd, mt.lvd, dsgn, Mb, bpart, bcnt);
      else
        FMMPC_CUDA(cudaMemsetAsync(Mb, 0, sizeof(cpx<R>) * P * g.nbcell * nrhs, s));
    }
    FMMPC_LAUNCH_CHECK();
    ++launches;
  }
  // with the tensor-core M2L (L >= 2) the boundary-source part of the volume locals is kept
  // apart for the downward pass to add, so it can run while the volume M2L still runs
  const bool vbv_sep = std::is_same<R, float>::value && H.tcm.enabled && with_bnd && Ls.n_vbv_cells > 0;
  auto run_vbv_sep = [&]() {
    k_m2l_vbv<R, P><<<nblk(Ls.n_vbv_cells * nrhs * 8), 256, 0, s>>>(gd, g.ncell, g.nbcell, nrhs, Ls.vbv_first,
                                                                     Ls.vbv_src, Mb, Lv, Ls.vbv_cells,
                                                                     Ls.n_vbv_cells, (cpx<R> *)H.fb.Lvb);
    FMMPC_LAUNCH_CHECK();
    ++launches;
  };
  if (side) {
    if (vbv_sep) run_vbv_sep();
    FMMPC_CUDA(cudaEventRecord(H.sev[2], ss));
    FMMPC_CUDA(cudaStreamWaitEvent(s, H.sev[2], 0));
    if (m2l_side) FMMPC_CUDA(cudaStreamWaitEvent(s, H.sev[5], 0));
  }
  mark(5);
  if (std::is_same<R, float>::value && H.tcm.enabled) {
    // volume-to-volume M2L on the tensor cores (mixed forms); boundary sources added after
    if (!m2l_side) launches += run_m2l_tc(H, Mv, Lv, nrhs, s);
    mark(6);
    if (vbv_sep && !side) run_vbv_sep();
  } else {
    k_m2l_vol<R, P><<<nblk(g.ncell * nrhs * 32), 256, 0, s>>>(gd, g.ncell, g.nbcell, nrhs, 1, with_bnd ? 1 : 0, 0,
                                                             Ls.m2l_first, Ls.m2l_src, Ls.vbv_first, Ls.vbv_src,
                                                             Mv, Mb, Lv);
    ++launches;
    mark(6);  // closes the M2L stage (its boundary sources are inside this kernel)
  }
  if (g.L < 2) {  // else the downward kernel adds the root constant
    k_root_const<R><<<1, 32, 0, s>>>(P, g.ncell, g.nbcell, nrhs, g.lnh, with_bnd ? 2 : 1, Mv, Mb, Lv, Lb);
    FMMPC_LAUNCH_CHECK();
    launches += 1;
  }
  mark(7);
  if (g.L < 2) launches += run_l2l<R, P>(H, nrhs, s);  // else L2L runs with L2P below
  if (!side && with_bnd && Ls.nbnear > 0) {
    mark(8);
    launches += run_bnd_near<R>(H, nrhs, s);
  }
  mark(9);
  const int do_bnd = (with_bnd && Ls.nbnear > 0) ? 1 : 0;
  const float *n1 = nullptr, *n2 = nullptr;
  if (tc) {
    if (!side) launches += run_p2p_tc(H, false, out, nrhs, s);
    n1 = H.tcp.near1;
    n2 = H.tcp.near2;
  } else {
    run_p2p<R>(H, H.fb.table, out, nrhs, s);  // writes the near field into out
    ++launches;
  }
  if (side && Ls.nbnear > 0) FMMPC_CUDA(cudaStreamWaitEvent(s, H.sev[4], 0));
  mark(10);
  if (g.L >= 2) run_downward<R, P>(H, out, nrhs, do_bnd, with_bnd ? 1 : 0, s, n1, n2, vbv_sep);
  else run_far_final<R>(H, out, nrhs, do_bnd, s, n1, n2);
  ++launches;
  mark_end();
  H.launches = launches;
}

// Translation matrices from the paper's formulas in scaled form (double, then cast).
template <typename R>
void build_mats(fmmpc_handle &H, std::vector<cpx<R>> &out) {
  const Geo &g = H.g;
  const int P = g.p;
  typedef std::complex<double> C;
  static double bin[2 * MAXP + 2][2 * MAXP + 2];
  for (int a = 0; a < 2 * MAXP + 2; ++a)
    for (int b = 0; b < 2 * MAXP + 2; ++b)
      bin[a][b] = (b == 0) ? 1.0 : (a == 0 ? 0.0 : bin[a - 1][b - 1] + bin[a - 1][b]);
  auto powc = [](C z, int k) { C r(1, 0); for (int i = 0; i < k; ++i) r *= z; return r; };
  // M2M from a child at offset w in parent units with child scale = parent scale / sc:
  // T[0][0] = 1, T[n][0] = -w^n / n, T[n][k] = sc^{-k} w^{n-k} C(n-1, k-1)
  auto m2m = [&](C w, double sc, std::vector<C> &T) {
    T.assign(P * P, C(0, 0));
    T[0] = 1.0;
    for (int nn = 1; nn < P; ++nn) {
      T[nn * P] = -powc(w, nn) / (double)nn;
      for (int k = 1; k <= nn; ++k) T[nn * P + k] = std::pow(1.0 / sc, k) * powc(w, nn - k) * bin[nn - 1][k - 1];
    }
  };
  // L2L to a child at w: S[n][k] = 2^{-n} w^{k-n} C(k, n)
  auto l2l = [&](C w, std::vector<C> &S) {
    S.assign(P * P, C(0, 0));
    for (int nn = 0; nn < P; ++nn)
      for (int k = nn; k < P; ++k) S[nn * P + k] = std::pow(0.5, nn) * powc(w, k - nn) * bin[k][nn];
  };
  std::vector<C> all, T;
  for (int ch = 0; ch < 4; ++ch) {
    m2m(C((ch & 1) ? 0.25 : -0.25, (ch & 2) ? 0.25 : -0.25), 2.0, T);
    all.insert(all.end(), T.begin(), T.end());
  }
  for (int ch = 0; ch < 4; ++ch) {
    l2l(C((ch & 1) ? 0.25 : -0.25, (ch & 2) ? 0.25 : -0.25), T);
    all.insert(all.end(), T.begin(), T.end());
  }
  const int n = g.n;
  const C edir[4] = {C(1, 0), C(0, 1), C(-1, 0), C(0, -1)};
  const double ell = (n + 1.0) / n;
  // Element e of a run at scale rho about its midpoint: unit single layer Mt_0 = 2 a rho,
  // Mt_k = -2 e^k a^{k+1} rho / (k (k+1)) for even k (0 for odd), a = ell / (2 rho); unit
  // double layer (int_e dG/dn_y is -(1/2pi) Re of -i (log(z - b) - log(z - a)) with a, b
  // its ends in traversal order and the outward normal the tangent turned clockwise: point
  // weights -i at b, +i at a; no factor h, a closed element run being scale free): Mt_0 = 0,
  // Mt_k = 2 i e^k a^k / k for odd k (0 for even); unit point source at the midpoint (the
  // transpose pass): Mt = (1, 0, ...); each shifted to the run centre at equal scale.  The
  // tables are formed for the run of every level l of the boundary tree, at that level's
  // scale n >> l: since M2M is exact, each level's multipoles follow directly from the
  // element densities, with no pass from level to level.
  for (int kind = 0; kind < 3; ++kind)
    for (int l = 0; l <= g.L; ++l) {
      const int len = n >> l;
      const double rl = len, al = ell / (2.0 * rl);
      for (int sd = 0; sd < 4; ++sd)
        for (int e = 0; e < len; ++e) {
          std::vector<C> el(P, C(0, 0));
          if (kind == 0) {
            el[0] = 2.0 * al * rl;
            for (int k = 2; k < P; k += 2) el[k] = -2.0 * powc(edir[sd], k) * std::pow(al, k + 1) * rl / (k * (k + 1.0));
          } else if (kind == 1) {
            for (int k = 1; k < P; k += 2) el[k] = C(0.0, 2.0) * powc(edir[sd], k) * std::pow(al, k) / (double)k;
          } else {
            el[0] = 1.0;
          }
          m2m(((e + 0.5 - 0.5 * len) * ell / rl) * edir[sd], 1.0, T);
          for (int nn = 0; nn < P; ++nn) {
            C v(0, 0);
            for (int k = 0; k <= nn; ++k) v += T[nn * P + k] * el[k];
            all.push_back(v);
          }
        }
    }
  out.resize(all.size());
  for (size_t i = 0; i < all.size(); ++i) out[i] = mk<R>((R)all[i].real(), (R)all[i].imag());
}

template <typename R>
void alloc_fmm(fmmpc_handle &H) {
  Geo &g = H.g;
  const int nr = H.nrhs_max;
  H.fb.wpad = H.pool.get<R>((size_t)nr * g.npad * g.npad);
  FMMPC_CUDA(cudaMemsetAsync(H.fb.wpad, 0, sizeof(R) * (size_t)nr * g.npad * g.npad, H.stream));
  H.fb.Mv = H.pool.get<cpx<R>>((size_t)nr * g.ncell * g.p);
  H.fb.up_ncount = std::max<int64_t>(1, level_offset(std::max(g.L - 3, 1)));
  H.fb.up_count = H.pool.get<int>((size_t)nr * H.fb.up_ncount);
  FMMPC_CUDA(cudaMemsetAsync(H.fb.up_count, 0, sizeof(int) * (size_t)nr * H.fb.up_ncount, H.stream));
  H.fb.Lv = H.pool.get<cpx<R>>((size_t)nr * g.ncell * g.p);
  H.fb.Mb = H.pool.get<cpx<R>>((size_t)nr * g.nbcell * g.p);
  H.fb.Lb = H.pool.get<cpx<R>>((size_t)nr * g.nbcell * g.p);
  H.fb.phib = H.pool.get<R>((size_t)nr * std::max<int64_t>(1, H.lists.nbnear) * g.m * g.m);
  H.fb.vcol = H.pool.get<double>((size_t)nr * g.NG);
  H.fb.q = H.pool.get<double>((size_t)nr * g.NG);
  H.fb.vt = H.pool.get<double>((size_t)nr * g.NG);
  H.fb.Lvb = H.pool.get<cpx<R>>((size_t)nr * std::max<int64_t>(1, H.lists.n_vbv_cells) * g.p);
  H.fb.vnear = H.pool.get<R>((size_t)nr * g.NG);
  // boundary upward pass: chunk partials and arrival counts of the coarse levels (cells of
  // more than BUP_CHUNK elements)
  H.fb.bup_lc = 0;
  while ((g.n >> H.fb.bup_lc) > BUP_CHUNK && H.fb.bup_lc < g.L) ++H.fb.bup_lc;
  const int64_t ncc = std::max<int64_t>(1, blevel_offset(H.fb.bup_lc));
  H.fb.bup_part = H.pool.get<cpx<R>>((size_t)nr * bup_blocks(g.n, g.L) * g.p);
  H.fb.bup_cnt = H.pool.get<int>((size_t)nr * ncc);
  FMMPC_CUDA(cudaMemsetAsync(H.fb.bup_cnt, 0, sizeof(int) * (size_t)nr * ncc, H.stream));
  if (std::is_same<R, float>::value) {  // two-word FP32 BEM apply
    H.fb.vt_hi = H.pool.get<float>((size_t)nr * g.NG);
    H.fb.vt_lo = H.pool.get<float>((size_t)nr * g.NG);
  }
  std::vector<cpx<R>> mats;
  build_mats<R>(H, mats);
  H.fb.mats = H.pool.get<cpx<R>>(mats.size());
  FMMPC_CUDA(cudaMemcpyAsync(H.fb.mats, mats.data(), sizeof(cpx<R>) * mats.size(), cudaMemcpyHostToDevice, H.stream));
  // lattice table, rows dy = 0..Rn (the table is even in dy), columns dx at c0 + Rn + dx;
  // stride chosen so that consecutive rows start 16 bytes apart modulo the 128-byte bank window
  const int Rn = g.R * g.m + g.m - 1;
  const int c0 = ((g.m - 1 - Rn) % 4 + 4) % 4;
  int TS = c0 + 2 * Rn + 2;
  while ((TS * (int)sizeof(R)) % 128 != 16) ++TS;
  H.fb.Rn = Rn;
  H.fb.table_c0 = c0;
  H.fb.table_stride = TS;
  H.fb.table_rows = Rn + 1;
  const double cself = -0.5 * std::log(2.0) - 1.5 + 0.25 * PI;  // mean of ln|x| on the unit cell
  std::vector<R> t0((size_t)(Rn + 1) * TS, R(0)), t1((size_t)(Rn + 1) * TS, R(0));
  for (int dy = 0; dy <= Rn; ++dy)
    for (int dx = -Rn; dx <= Rn; ++dx) {
      const double v = (dx == 0 && dy == 0) ? cself : 0.5 * std::log((double)dx * dx + (double)dy * dy);
      t0[(size_t)dy * TS + c0 + Rn + dx] = (R)v;
      t1[(size_t)dy * TS + c0 + Rn + dx] = (R)(v + g.lnh);
    }
  H.fb.table = H.pool.get<R>(t0.size());
  H.fb.table_lnh = H.pool.get<R>(t1.size());
  FMMPC_CUDA(cudaMemcpyAsync(H.fb.table, t0.data(), sizeof(R) * t0.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(H.fb.table_lnh, t1.data(), sizeof(R) * t1.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
}

template <typename R>
void dispatch_apply(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  switch (H.g.p) {
    case 4: apply_impl<R, 4>(H, part, r, out, nrhs); break;
    case 6: apply_impl<R, 6>(H, part, r, out, nrhs); break;
    case 8: apply_impl<R, 8>(H, part, r, out, nrhs); break;
    case 10: apply_impl<R, 10>(H, part, r, out, nrhs); break;
    case 12: apply_impl<R, 12>(H, part, r, out, nrhs); break;
    case 16: apply_impl<R, 16>(H, part, r, out, nrhs); break;
    default: throw Error(FMMPC_ERR_UNSUPPORTED, "expansion order p must be one of 4, 6, 8, 10, 12, 16");
  }
}

}  // namespace

void init_fmm(fmmpc_handle &H) {
  const int side = 1 << H.g.L;
  const int m = H.g.m;
  int tx = (m == 16) ? 4 : 8, ty = (m == 4) ? 8 : 4;
  tx = std::min(tx, side);
  ty = std::min(ty, side);
  // the CUDA-core near field: on small grids, smaller tiles until there are two CTAs per SM
  // (down to 2 x 2 leaves), so that a 512^2 or 256^2 grid does not leave SMs idle
  int dev = 0, nsm = 0;
  FMMPC_CUDA(cudaGetDevice(&dev));
  FMMPC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  while ((int64_t)(side / tx) * (side / ty) < 2 * (int64_t)nsm && (tx > 2 || ty > 2)) {
    if (tx >= ty) tx /= 2;
    else ty /= 2;
  }
  H.tile_x = tx;
  H.tile_y = ty;
  if (H.prec == FMMPC_PREC_FP64) {
    if (m == 16) throw Error(FMMPC_ERR_UNSUPPORTED, "FP64 mode supports leaf side 4 or 8");
    set_p2p_smem_limit<double>();
    alloc_fmm<double>(H);
  } else {
    set_p2p_smem_limit<float>();
    alloc_fmm<float>(H);
    // near-boundary operators formed once (the geometry is fixed): element integrals at the
    // nodes of volume leaves next to the boundary, and the log kernel at collocation points
    const int64_t nent = H.lists.n_p2p_vb * (int64_t)H.g.m * H.g.m * H.g.m;
    if (nent > 0 && H.lists.nbnear > 0) {
      H.fb.knear = H.pool.get<float>(nent);
      H.fb.kcol = H.pool.get<float>(nent);
      k_bnd_near_mat<<<(unsigned)H.lists.nbnear, 256, 0, H.stream>>>(H.g, H.lists.nbnear, H.lists.pbv_leaf,
                                                                    H.lists.pbv_first, H.lists.pbv_src, H.fb.knear);
      k_colloc_mat<<<nblk((int64_t)H.g.NG * 32, 128), 128, 0, H.stream>>>(H.g, H.lists.pvb_first, H.lists.pvb_src,
                                                                         H.fb.kcol);
      FMMPC_LAUNCH_CHECK();
      FMMPC_CUDA(cudaStreamSynchronize(H.stream));
    }
  }
  // Stream priorities (copied into the kernel nodes of captured graphs, which are
  // instantiated to use them): the apply's critical chain (weights, upward pass, boundary
  // chain, downward pass) runs on the graph stream at the highest priority; the near-
  // boundary correction, which joins later, in between; the near field and the volume M2L,
  // which have slack, at the lowest, so that their many CTAs do not hold back the chain's
  // latency-bound kernels.
  int prio_low = 0, prio_high = 0;
  FMMPC_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  FMMPC_CUDA(cudaStreamCreateWithPriority(&H.gstream, cudaStreamNonBlocking, prio_high));
  FMMPC_CUDA(cudaEventCreateWithFlags(&H.gev_in, cudaEventDisableTiming));
  FMMPC_CUDA(cudaEventCreateWithFlags(&H.gev_out, cudaEventDisableTiming));
  FMMPC_CUDA(cudaStreamCreateWithPriority(&H.sstream, cudaStreamNonBlocking, prio_low));
  FMMPC_CUDA(cudaStreamCreateWithPriority(&H.sstream2, cudaStreamNonBlocking, (prio_low + prio_high) / 2));
  FMMPC_CUDA(cudaStreamCreateWithPriority(&H.sstream3, cudaStreamNonBlocking, prio_low));
  for (auto &e : H.sev) FMMPC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

namespace {

void apply_direct(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  if (H.prec == FMMPC_PREC_FP64) dispatch_apply<double>(H, part, r, out, nrhs);
  else dispatch_apply<float>(H, part, r, out, nrhs);
}

// The full apply replayed from a CUDA graph captured on the handle's internal stream, one
// graph per (r, z, n_rhs, timing) seen; the internal stream is ordered after and before
// the caller's stream with events, so the call keeps the stream semantics of the ABI.
void apply_graph(fmmpc_handle &H, const double *r, double *out, int nrhs) {
  GraphEntry *hit = nullptr;
  for (auto &e : H.gcache)
    if (e.r == r && e.out == out && e.nrhs == nrhs && e.timing == H.timing) hit = &e;
  if (!hit) {
    if (H.gcache.size() >= 64) {
      auto old = std::min_element(H.gcache.begin(), H.gcache.end(),
                                  [](const GraphEntry &a, const GraphEntry &b) { return a.last < b.last; });
      cudaGraphExecDestroy(old->exec);
      H.gcache.erase(old);
    }
    cudaStream_t user = H.stream;
    H.stream = H.gstream;
    cudaGraph_t graph = nullptr;
    FMMPC_CUDA(cudaStreamBeginCapture(H.gstream, cudaStreamCaptureModeThreadLocal));
    try {
      apply_direct(H, PART_FULL, r, out, nrhs);
    } catch (...) {
      cudaStreamEndCapture(H.gstream, &graph);
      if (graph) cudaGraphDestroy(graph);
      H.stream = user;
      throw;
    }
    H.stream = user;
    FMMPC_CUDA(cudaStreamEndCapture(H.gstream, &graph));
    GraphEntry e{r, out, nrhs, H.timing, nullptr, 0};
    cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    FMMPC_CUDA(ie);
    H.gcache.push_back(e);
    hit = &H.gcache.back();
  }
  hit->last = ++H.gclock;
  FMMPC_CUDA(cudaEventRecord(H.gev_in, H.stream));
  FMMPC_CUDA(cudaStreamWaitEvent(H.gstream, H.gev_in, 0));
  FMMPC_CUDA(cudaGraphLaunch(hit->exec, H.gstream));
  FMMPC_CUDA(cudaEventRecord(H.gev_out, H.gstream));
  FMMPC_CUDA(cudaStreamWaitEvent(H.stream, H.gev_out, 0));
}

}  // namespace

void apply_fmm_eager(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  apply_direct(H, part, r, out, nrhs);
}

void apply_fmm(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  if (part == PART_FULL && H.graphs) apply_graph(H, r, out, nrhs);
  else apply_direct(H, part, r, out, nrhs);
}

// ====================================================================== no-allocation variant
// Near field of V r computed with scratch that lives in a static device array instead of
// memory from cudaMalloc (see fmmpc_near_field_noalloc in fmmpc.h).  The array holds the
// log table followed by the zero-padded FP32 weight image; every call rewrites both.
namespace {

constexpr int64_t NOALLOC_FLOATS = int64_t(4) * 1024 * 1024;  // 16 MiB of FP32
constexpr int NOALLOC_MAX_DEVICES = 64;

__global__ void k_noalloc_table(float *__restrict__ tab, int Rn, int TS, int c0, double lnh) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)(Rn + 1) * TS) return;
  const int dy = (int)(k / TS), dx = (int)(k % TS) - c0 - Rn;
  float v = 0.0f;  // padding columns are read by the vector loads but never used
  if (dx >= -Rn && dx <= Rn) {
    const double cself = -0.5 * log(2.0) - 1.5 + 0.25 * PI;
    const double lg = (dx == 0 && dy == 0) ? cself : 0.5 * log((double)dx * dx + (double)dy * dy);
    v = (float)(lg + lnh);
  }
  tab[k] = v;
}

__global__ void k_noalloc_image(float *__restrict__ img, int n, int npad, int pad, double h2,
                                const double *__restrict__ r) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)npad * npad) return;
  const int y = (int)(k / npad) - pad, x = (int)(k % npad) - pad;
  img[k] = (x >= 0 && y >= 0 && x < n && y < n) ? (float)(h2 * r[(int64_t)y * n + x]) : 0.0f;
}

}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

namespace {

// Identity of the current CUDA context (unique for the life of the process), through the
// driver's cuCtxGetId reached via the runtime's entry-point query; 0 if unavailable.
unsigned long long current_ctx_id() {
  using ctx_id_fn = int (*)(void *, unsigned long long *);
  static ctx_id_fn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<ctx_id_fn>(f);
  }();
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != 0) return 0;
  return id;
}

// Device address of g_noalloc_scratch, resolved once per device and context: a context
// made anew (after cudaDeviceReset) reloads the module, and the array may then sit at a
// different address, so the cached address is taken again when the context id changes.
cudaError_t noalloc_scratch(float **out) {
  static std::mutex mu;
  static float *ptr[NOALLOC_MAX_DEVICES] = {};
  static unsigned long long ctx[NOALLOC_MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long id = current_ctx_id();  // 0: no current context yet, or no query
  if (!ptr[dev] || id == 0 || id != ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the primary context current if needed
    if (e != cudaSuccess) return e;
    ptr[dev] = static_cast<float *>(p);
    ctx[dev] = id ? id : current_ctx_id();
  }
  *out = ptr[dev];
  return cudaSuccess;
}

// Dynamic shared memory the near-field kernel of leaf side M may take on this device (the
// per-block opt-in maximum minus its static use).
template <int M>
cudaError_t noalloc_smem_cap(size_t *cap) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, k_p2p<float, M>);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  *cap = (size_t)optin - fa.sharedSizeBytes;
  return cudaSuccess;
}

// The attribute is per function and shared with the handle-based near field, so it is only
// ever raised, never set below what another caller configured.
template <int M>
cudaError_t noalloc_launch(const P2PArgs<float> &a, int L, size_t smem, cudaStream_t s) {
  const int side = 1 << L;
  dim3 grid(side / a.tile_x, side / a.tile_y, 1);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, k_p2p<float, M>);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes < smem) {
    e = cudaFuncSetAttribute(k_p2p<float, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_p2p<float, M><<<grid, a.tile_x * a.tile_y * M, smem, s>>>(a);
  return cudaPeekAtLastError();
}

}  // namespace

int near_field_noalloc(int32_t n, double side, int32_t leaf_max, double theta, const double *r_dev,
                       double *out_dev, void *stream) {
  if (!r_dev || !out_dev || r_dev == out_dev) return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: r and out must be distinct device buffers");
  if (n < 4 || n > 4096 || (n & (n - 1)) != 0) return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: n must be a power of two in [4, 4096]");
  if (!(side > 0.0) || !(theta > 0.0 && theta < 1.0) || leaf_max < 16)
    return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: need side > 0, 0 < theta < 1, leaf_max >= 16");
  int L = 0, m = n;
  while ((int64_t)m * m > leaf_max) { m /= 2; ++L; }
  if (m != 4 && m != 8 && m != 16) return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: leaf side must be 4, 8 or 16");
  // P2P stencil of a uniform tree: leaf offsets o with 2 tden^2 >= tnum^2 |o|^2 (the pair and
  // all its ancestor pairs fail the MAC), the same set the dual tree traversal produces
  const int tn = (int)std::lround(theta * 1000.0), td = 1000;
  Stencil st{};
  int R = 0;
  for (int oy = -16; oy <= 16; ++oy)
    for (int ox = -16; ox <= 16; ++ox)
      if (2LL * td * td >= (long long)tn * tn * (ox * ox + oy * oy)) R = std::max(R, std::max(std::abs(ox), std::abs(oy)));
  if (R >= 16) return set_global_error(FMMPC_ERR_UNSUPPORTED, "near_field_noalloc: theta too small (stencil radius above 15 leaves)");
  st.R = R;
  for (int oy = -R; oy <= R; ++oy) {
    int lo = 1, hi = 0;
    for (int ox = -R; ox <= R; ++ox)
      if (2LL * td * td >= (long long)tn * tn * (ox * ox + oy * oy)) {
        if (lo > hi) lo = ox;
        hi = ox;
        ++st.count;
      }
    st.ox0[oy + R] = lo;
    st.ox1[oy + R] = hi;
  }
  const int pad = R * m, npad = n + 2 * pad, Rn = R * m + m - 1;
  const int c0 = ((m - 1 - Rn) % 4 + 4) % 4;
  int TS = c0 + 2 * Rn + 2;
  while ((TS * 4) % 128 != 16) ++TS;
  const int64_t tab_floats = (int64_t)(Rn + 1) * TS;
  const int64_t need = tab_floats + (int64_t)npad * npad;
  if (need > NOALLOC_FLOATS)
    return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: grid too large for the 16 MiB static scratch (n = 1024 with 8x8 leaves and theta 0.4 is the largest such grid)");
  const int sidel = 1 << L;
  int tx = (m == 16) ? 4 : 8, ty = (m == 4) ? 8 : 4;
  tx = std::min(tx, sidel);
  ty = std::min(ty, sidel);
  const int HX = (tx + 2 * R) * m, HY = (ty + 2 * R) * m;
  const size_t smem = ((size_t)HY * HX + (size_t)(Rn + 1) * TS) * sizeof(float);
  size_t cap = 0;
  cudaError_t e = (m == 4) ? noalloc_smem_cap<4>(&cap) : (m == 8) ? noalloc_smem_cap<8>(&cap) : noalloc_smem_cap<16>(&cap);
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  if (smem > cap)  // checked before any work is queued
    return set_global_error(FMMPC_ERR_UNSUPPORTED, "near_field_noalloc: the source tile of this theta and leaf size does not fit in one block's shared memory");
  float *scratch = nullptr;
  e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const double h = side / (n + 1);
  float *tab = scratch, *img = scratch + tab_floats;  // tab_floats is a multiple of 4: 16-byte aligned image
  k_noalloc_table<<<(unsigned)((tab_floats + 255) / 256), 256, 0, s>>>(tab, Rn, TS, c0, std::log(h));
  k_noalloc_image<<<(unsigned)(((int64_t)npad * npad + 255) / 256), 256, 0, s>>>(img, n, npad, pad, h * h, r_dev);
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  P2PArgs<float> a{};
  a.wpad = img; a.table = tab; a.out = out_dev;
  a.n = n; a.npad = npad; a.L = L; a.R_ = R; a.Rn = Rn;
  a.HX = HX; a.HY = HY; a.TS = TS; a.c0 = c0;
  a.tile_x = tx; a.tile_y = ty; a.nrhs = 1;
  a.st = st;
  switch (m) {
    case 4: e = noalloc_launch<4>(a, L, smem, s); break;
    case 8: e = noalloc_launch<8>(a, L, smem, s); break;
    default: e = noalloc_launch<16>(a, L, smem, s); break;
  }
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  return FMMPC_OK;
}

}  // namespace fmmpc
