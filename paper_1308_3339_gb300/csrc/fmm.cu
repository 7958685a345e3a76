// The preconditioner apply z = P^{-1} r (Sec. 3.2 Fig. f:flow_chart) on the GPU.
//
// Pass A (volume sources w = h^2 r):  P2M at the leaves, M2M up the quadtree (Sec. 5.3
//   items 1-2); M2L from volume cells into the boundary cells, L2L along each side, L2P
//   plus the near field at the collocation points: (V r)(y_m), the right-hand side of
//   Eq. e:ubound with z = 0 on Gamma.  q = S^{-1}(-(V r)|_Gamma) in FP64 (Sec. 4.3).
// Pass B: boundary elements carrying q become sources (exact segment multipoles), M2M up
//   the boundary trees; one M2L over volume and boundary sources into the volume locals
//   (item 3), L2L down (item 4); the final kernel sums the lattice near field (P2P),
//   L2P (item 5) and the closed-form near integrals of the elements: Eq. e:uinter.
//
// Everything runs in node units with scaled expansions (see common.cuh).  The near field
// uses the lattice: G between two nodes depends only on their integer offset, so P2P is
// a block convolution of the weight image with a table of ln|d| over the stencil of
// leaf offsets that the dual tree traversal produced.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "handle.cuh"

namespace fmmpc {

__constant__ double c_binom[MAXP + 1][MAXP + 1];

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

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
// Mt_0 = sum w_j, Mt_k = -sum w_j zt_j^k / k, zt_j = (z_j - c) / rho_L.  Warp per leaf.
template <typename R>
__global__ void k_p2m_leaf(Geo g, int nrhs, const R *__restrict__ wpad, cpx<R> *__restrict__ Mv) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= g.nleaf * nrhs) return;
  const int rhs = (int)(wid / g.nleaf);
  const uint32_t c = (uint32_t)(wid % g.nleaf);
  int a, b;
  morton_decode(c, a, b);
  const int m = g.m, p = g.p;
  const R *W = wpad + (int64_t)rhs * g.npad * g.npad;
  const R half = R(0.5) * (m - 1), invm = R(1) / m;
  cpx<R> acc[MAXP];
#pragma unroll
  for (int k = 0; k < MAXP; ++k) acc[k] = mk<R>(0, 0);
  for (int t = lane; t < m * m; t += 32) {
    int i = t % m, j = t / m;
    R w = W[(int64_t)(b * m + j + g.pad) * g.npad + a * m + i + g.pad];
    cpx<R> z = mk<R>((i - half) * invm, (j - half) * invm), pw = z;
    acc[0].re += w;
#pragma unroll
    for (int k = 1; k < MAXP; ++k)
      if (k < p) {
        R s = -w / k;
        acc[k].re = fma(s, pw.re, acc[k].re);
        acc[k].im = fma(s, pw.im, acc[k].im);
        pw = pw * z;
      }
  }
  cpx<R> *out = Mv + (int64_t)rhs * g.ncell * p + (level_offset(g.L) + c) * p;
#pragma unroll
  for (int k = 0; k < MAXP; ++k)
    if (k < p) {
      R re = warp_sum(acc[k].re), im = warp_sum(acc[k].im);
      if (lane == 0) out[k] = mk(re, im);
    }
}

// ------------------------------------------------------------------ M2M (item 2)
// Child at w = (c_child - c_parent)/rho_P = (+-1/4, +-1/4), rho_child = rho_P / 2:
// Mt_n(P) = -Mt_0 w^n/n + sum_{k=1}^n Mt_k(child) 2^{-k} w^{n-k} C(n-1, k-1).
template <typename R>
__global__ void k_m2m_vol(int l, int p, int64_t ncell, int nrhs, cpx<R> *__restrict__ Mv) {
  const int64_t nc = int64_t(1) << (2 * l);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nrhs) return;
  const int rhs = (int)(t / nc);
  const int64_t c = t % nc;
  cpx<R> *M = Mv + (int64_t)rhs * ncell * p;
  cpx<R> acc[MAXP];
  for (int k = 0; k < p; ++k) acc[k] = mk<R>(0, 0);
  for (int ch = 0; ch < 4; ++ch) {
    const cpx<R> *Mc = M + (level_offset(l + 1) + 4 * c + ch) * p;
    cpx<R> w = mk<R>((ch & 1) ? R(0.25) : R(-0.25), (ch & 2) ? R(0.25) : R(-0.25));
    cpx<R> wp[MAXP], m[MAXP];
    wp[0] = mk<R>(1, 0);
    for (int k = 1; k < p; ++k) wp[k] = wp[k - 1] * w;
    for (int k = 0; k < p; ++k) m[k] = Mc[k];
    acc[0] = acc[0] + m[0];
    for (int nn = 1; nn < p; ++nn) {
      cpx<R> v = (R(-1) / nn) * (m[0] * wp[nn]);
      R two = 1;
      for (int k = 1; k <= nn; ++k) {
        two *= R(0.5);
        v = v + (two * (R)c_binom[nn - 1][k - 1]) * (m[k] * wp[nn - k]);
      }
      acc[nn] = acc[nn] + v;
    }
  }
  cpx<R> *out = M + (level_offset(l) + c) * p;
  for (int k = 0; k < p; ++k) out[k] = acc[k];
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
  R invf = 1;
#pragma unroll
  for (int k = 1; k < P; ++k) {
    a[k] = invf * m[k];
    invf = invf / R(k);
  }
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

template <typename R, int P>
__device__ __forceinline__ void m2l_finish(cpx<R> (&H)[P], int lane, cpx<R> *__restrict__ out) {
  R f = 1;
#pragma unroll
  for (int n = 0; n < P; ++n) {
    if (n > 0) f = -f / R(n);
    R re = warp_sum(H[n].re), im = warp_sum(H[n].im);
    if (lane == 0) out[n] = mk(f * re, f * im);
  }
}

// Volume targets: warp per (cell, rhs) over all cells of all levels; volume sources
// from the M2L list and, when with_bnd, boundary sources from the volume-boundary list.
template <typename R, int P>
__global__ void k_m2l_vol(GeoDev gd, int64_t ncell, int64_t nbcell, int nrhs, int with_bnd,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                          const int32_t *__restrict__ bfirst, const int32_t *__restrict__ bsrc,
                          const cpx<R> *__restrict__ Mv, const cpx<R> *__restrict__ Mb,
                          cpx<R> *__restrict__ Lv) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= ncell * nrhs) return;
  const int rhs = (int)(wid / ncell);
  const int64_t gidx = wid % ncell;
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
  const cpx<R> *M = Mv + (int64_t)rhs * ncell * P + level_offset(l) * P;
  for (int e = first[gidx] + lane; e < first[gidx + 1]; e += 32) {
    const uint32_t s = (uint32_t)src[e];
    int sx, sy;
    morton_decode(s, sx, sy);
    m2l_accum<R, P>(H, M + (int64_t)s * P, mk<R>((R)(tx - sx), (R)(ty - sy)), lnrho);
  }
  if (with_bnd) {
    int64_t X, Y, sw;
    vol_geom(gd, l, c, X, Y, sw);
    X <<= gd.L;
    Y <<= gd.L;
    const double scale = 1.0 / ((double)rho * (double)(int64_t(1) << (gd.L + 1)));
    const cpx<R> *MB = Mb + (int64_t)rhs * nbcell * P + blevel_offset(l) * P;
    for (int e = bfirst[gidx] + lane; e < bfirst[gidx + 1]; e += 32) {
      const uint32_t b = (uint32_t)bsrc[e];
      int64_t BX, BY, bs;
      bnd_geom(gd, l, b, BX, BY, bs);
      m2l_accum<R, P>(H, MB + (int64_t)b * P,
                      mk<R>((R)((double)(X - BX) * scale), (R)((double)(Y - BY) * scale)), lnrho);
    }
  }
  m2l_finish<R, P>(H, lane, Lv + (int64_t)rhs * ncell * P + gidx * P);
}

// Boundary targets (pass A): warp per (boundary cell, rhs); volume sources.
template <typename R, int P>
__global__ void k_m2l_bnd(GeoDev gd, int64_t ncell, int64_t nbcell, int nrhs,
                          const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                          const cpx<R> *__restrict__ Mv, cpx<R> *__restrict__ Lb) {
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
  const double scale = 1.0 / ((double)rho * (double)(int64_t(1) << (gd.L + 1)));
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
                    mk<R>((R)((double)(BX - X) * scale), (R)((double)(BY - Y) * scale)), lnrho);
  }
  m2l_finish<R, P>(H, lane, Lb + (int64_t)rhs * nbcell * P + gb * P);
}

// ------------------------------------------------------------------ L2L (item 4)
// Lt_n(child) += 2^{-n} sum_{k=n}^{p-1} Lt_k(parent) w^{k-n} C(k, n),
// w = (c_child - c_parent) / rho_P.
template <typename R>
__device__ __forceinline__ void l2l_add(int p, const cpx<R> *__restrict__ Lp, cpx<R> w,
                                        cpx<R> *__restrict__ Lc) {
  cpx<R> wp[MAXP], lp[MAXP];
  wp[0] = mk<R>(1, 0);
  for (int k = 1; k < p; ++k) wp[k] = wp[k - 1] * w;
  for (int k = 0; k < p; ++k) lp[k] = Lp[k];
  R two = 1;
  for (int nn = 0; nn < p; ++nn) {
    cpx<R> v = mk<R>(0, 0);
    for (int k = nn; k < p; ++k) v = v + (R)c_binom[k][nn] * (lp[k] * wp[k - nn]);
    Lc[nn] = Lc[nn] + two * v;
    two *= R(0.5);
  }
}

template <typename R>
__global__ void k_l2l_vol(int l, int p, int64_t ncell, int nrhs, cpx<R> *__restrict__ Lv) {
  const int64_t nc = int64_t(1) << (2 * (l + 1));
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nrhs) return;
  const int rhs = (int)(t / nc);
  const int64_t cc = t % nc;
  const int ch = (int)(cc & 3);
  cpx<R> *Lx = Lv + (int64_t)rhs * ncell * p;
  cpx<R> w = mk<R>((ch & 1) ? R(0.25) : R(-0.25), (ch & 2) ? R(0.25) : R(-0.25));
  l2l_add<R>(p, Lx + (level_offset(l) + (cc >> 2)) * p, w, Lx + (level_offset(l + 1) + cc) * p);
}

__device__ __forceinline__ void side_dir(int side, double &ex, double &ey) {
  ex = (side == 0) ? 1.0 : (side == 2 ? -1.0 : 0.0);
  ey = (side == 1) ? 1.0 : (side == 3 ? -1.0 : 0.0);
}
// point at arclength t (node units) along side `side` of the boundary square [0, n+1]^2
__device__ __forceinline__ void side_point(int side, double t, double np1, double &x, double &y) {
  switch (side) {
    case 0: x = t; y = 0; break;
    case 1: x = np1; y = t; break;
    case 2: x = np1 - t; y = np1; break;
    default: x = 0; y = np1 - t; break;
  }
}

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

// boundary child run at level l+1 from its parent at level l: w = (2j-1)(n+1)/(4n) e_side
template <typename R>
__global__ void k_l2l_bnd(int l, int n, int p, int64_t nbcell, int nrhs, cpx<R> *__restrict__ Lb) {
  const int64_t nc = 4 * (int64_t(1) << (l + 1));
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nrhs) return;
  const int rhs = (int)(t / nc);
  const int64_t id = t % nc;
  const int side = (int)(id >> (l + 1));
  const int64_t kc = id & ((int64_t(1) << (l + 1)) - 1);
  const int j = (int)(kc & 1);
  double ex, ey;
  side_dir(side, ex, ey);
  const double f = (2 * j - 1) * (n + 1.0) / (4.0 * n);
  cpx<R> *Lx = Lb + (int64_t)rhs * nbcell * p;
  const int64_t parent = ((int64_t)side << l) + (kc >> 1);
  l2l_add<R>(p, Lx + (blevel_offset(l) + parent) * p, mk<R>((R)(f * ex), (R)(f * ey)),
             Lx + (blevel_offset(l + 1) + id) * p);
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

// ------------------------------------------------------------------ collocation points
// (V r)(y_m) = -(1/2pi)[ Re sum_n Lt_n zt^n  +  sum_{near nodes} w_j ln|y_m - x_j| ].
// Warp per (boundary leaf, rhs); m <= 16 collocation points per leaf.
template <typename R>
__global__ void k_colloc(Geo g, int nrhs, const R *__restrict__ wpad, const cpx<R> *__restrict__ Lb,
                         const int32_t *__restrict__ pfirst, const int32_t *__restrict__ psrc,
                         double *__restrict__ vcol) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= g.nbleaf * nrhs) return;
  const int rhs = (int)(wid / g.nbleaf);
  const int64_t bl = wid % g.nbleaf;
  const int n = g.n, m = g.m, L = g.L, p = g.p;
  const int side = (int)(bl >> L);
  const int64_t kk = bl & ((int64_t(1) << L) - 1);
  const double ell = (n + 1.0) / n;
  double ex, ey;
  side_dir(side, ex, ey);
  const R *W = wpad + (int64_t)rhs * g.npad * g.npad;
  R acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0;
  const R inv2n = R(1) / (R)(2 * n);
  for (int e0 = pfirst[bl]; e0 < pfirst[bl + 1]; ++e0) {
    int a, b;
    morton_decode((uint32_t)psrc[e0], a, b);
    for (int t = lane; t < m * m; t += 32) {
      const int i = a * m + t % m, j = b * m + t / m;
      const R w = W[(int64_t)(j + g.pad) * g.npad + i + g.pad];
      int u, d;
      side_coords(side, n + 1, i + 1, j + 1, u, d);
      const R dd = (R)d * (R)d;
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (e < m) {
          // (y_e - x) along the side = ((2(k m + e) + 1)(n + 1) - 2 u n) / (2n), exact numerator
          const int64_t num = (2 * (kk * m + e) + 1) * (int64_t)(n + 1) - 2 * (int64_t)u * n;
          const R ds = (R)num * inv2n;
          acc[e] += w * (R(0.5) * dev_log<R>(ds * ds + dd));
        }
    }
  }
  const cpx<R> *Lc = Lb + (int64_t)rhs * g.nbcell * p + (blevel_offset(L) + bl) * p;
#pragma unroll
  for (int e = 0; e < 16; ++e)
    if (e < m) {
      R s = warp_sum(acc[e]);
      if (lane == e) {
        const double off = (e + 0.5 - 0.5 * m) * ell / m;  // (y_e - c) / rho_L along the side
        cpx<R> z = mk<R>((R)(off * ex), (R)(off * ey)), v = mk<R>(0, 0);
        for (int k = p - 1; k >= 0; --k) v = v * z + Lc[k];
        vcol[(int64_t)rhs * g.NG + side * n + kk * m + e] = -((double)s + (double)v.re) / (2.0 * PI);
      }
    }
}

// ------------------------------------------------------------------ BEM solve (FP64)
// q = -S^{-1} (V r)|_Gamma with the inverse formed at set-up.  Warp per (row, rhs).
__global__ void k_bem_gemv(int NG, int nrhs, const double *__restrict__ Sinv,
                           const double *__restrict__ vcol, double *__restrict__ q) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)NG * nrhs) return;
  const int row = (int)(wid % NG), rhs = (int)(wid / NG);
  const double *S = Sinv + (int64_t)row * NG;
  const double *v = vcol + (int64_t)rhs * NG;
  double acc = 0.0;
  for (int k = lane; k < NG; k += 32) acc = fma(S[k], v[k], acc);
  acc = warp_sum(acc);
  if (lane == 0) q[(int64_t)rhs * NG + row] = -acc;
}

// ------------------------------------------------------------------ boundary P2M / M2M
// Element e of a leaf run: density q_e (physical) -> qt = q_e h per node-unit length.
// About its midpoint: Mt_0 = qt rho 2a, Mt_k = -qt rho 2 e^k a^{k+1} / (k (k+1)) for even
// k (0 for odd), a = half-length / rho; shifted to the run centre by the M2M formula at
// equal scale (w = (y_e - c) / rho, no 2^{-k}).
template <typename R>
__global__ void k_p2m_bnd(Geo g, int nrhs, const double *__restrict__ q, cpx<R> *__restrict__ Mb) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nbleaf * nrhs) return;
  const int rhs = (int)(t / g.nbleaf);
  const int64_t bl = t % g.nbleaf;
  const int n = g.n, m = g.m, L = g.L, p = g.p;
  const int side = (int)(bl >> L);
  const int64_t kk = bl & ((int64_t(1) << L) - 1);
  double ex, ey;
  side_dir(side, ex, ey);
  const double ell = (n + 1.0) / n, rho = m, a = ell / (2.0 * rho);
  const cpx<R> es = mk<R>((R)ex, (R)ey);
  cpx<R> acc[MAXP], el[MAXP], wp[MAXP];
  for (int k = 0; k < p; ++k) acc[k] = mk<R>(0, 0);
  for (int e = 0; e < m; ++e) {
    const double qr = q[(int64_t)rhs * g.NG + side * n + kk * m + e] * g.h * rho;
    el[0] = mk<R>((R)(qr * 2.0 * a), 0);
    cpx<R> ep = mk<R>(1, 0);
    double ak = a;
    for (int k = 1; k < p; ++k) {
      ep = ep * es;
      ak *= a;  // a^{k+1}
      el[k] = (k % 2 == 0) ? (R)(-qr * 2.0 * ak / (k * (k + 1.0))) * ep : mk<R>(0, 0);
    }
    const double off = (e + 0.5 - 0.5 * m) * ell / rho;
    const cpx<R> w = mk<R>((R)(off * ex), (R)(off * ey));
    wp[0] = mk<R>(1, 0);
    for (int k = 1; k < p; ++k) wp[k] = wp[k - 1] * w;
    acc[0] = acc[0] + el[0];
    for (int nn = 1; nn < p; ++nn) {
      cpx<R> v = (R(-1) / nn) * (el[0] * wp[nn]);
      for (int k = 1; k <= nn; ++k) v = v + (R)c_binom[nn - 1][k - 1] * (el[k] * wp[nn - k]);
      acc[nn] = acc[nn] + v;
    }
  }
  cpx<R> *out = Mb + (int64_t)rhs * g.nbcell * p + (blevel_offset(L) + bl) * p;
  for (int k = 0; k < p; ++k) out[k] = acc[k];
}

template <typename R>
__global__ void k_m2m_bnd(int l, int n, int p, int64_t nbcell, int nrhs, cpx<R> *__restrict__ Mb) {
  const int64_t nc = 4 * (int64_t(1) << l);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * nrhs) return;
  const int rhs = (int)(t / nc);
  const int64_t id = t % nc;
  const int side = (int)(id >> l);
  const int64_t k = id & ((int64_t(1) << l) - 1);
  double ex, ey;
  side_dir(side, ex, ey);
  cpx<R> *M = Mb + (int64_t)rhs * nbcell * p;
  cpx<R> acc[MAXP], wp[MAXP], mc[MAXP];
  for (int q = 0; q < p; ++q) acc[q] = mk<R>(0, 0);
  for (int j = 0; j < 2; ++j) {
    const int64_t child = ((int64_t)side << (l + 1)) + 2 * k + j;
    const cpx<R> *Mc = M + (blevel_offset(l + 1) + child) * p;
    const double f = (2 * j - 1) * (n + 1.0) / (4.0 * n);
    const cpx<R> w = mk<R>((R)(f * ex), (R)(f * ey));
    wp[0] = mk<R>(1, 0);
    for (int q = 1; q < p; ++q) wp[q] = wp[q - 1] * w;
    for (int q = 0; q < p; ++q) mc[q] = Mc[q];
    acc[0] = acc[0] + mc[0];
    for (int nn = 1; nn < p; ++nn) {
      cpx<R> v = (R(-1) / nn) * (mc[0] * wp[nn]);
      R two = 1;
      for (int q = 1; q <= nn; ++q) {
        two *= R(0.5);
        v = v + (two * (R)c_binom[nn - 1][q - 1]) * (mc[q] * wp[nn - q]);
      }
      acc[nn] = acc[nn] + v;
    }
  }
  cpx<R> *out = M + (blevel_offset(l) + id) * p;
  for (int q = 0; q < p; ++q) out[q] = acc[q];
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

// Warp per (volume leaf next to the boundary, rhs): phib = sum_k qt_k int_k ln|x - y| ds.
template <typename R>
__global__ void k_bnd_near(Geo g, int64_t nbnear, int nrhs, const int32_t *__restrict__ leaf,
                           const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                           const double *__restrict__ q, R *__restrict__ phib) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nbnear * nrhs) return;
  const int rhs = (int)(wid / nbnear);
  const int64_t slot = wid % nbnear;
  const int n = g.n, m = g.m, L = g.L;
  int a, b;
  morton_decode((uint32_t)leaf[slot], a, b);
  const R ell = (R)((n + 1.0) / n), invn = R(1) / (R)n, hR = (R)g.h;
  const double *qr = q + (int64_t)rhs * g.NG;
  for (int t = lane; t < m * m; t += 32) {
    const int x = a * m + t % m + 1, y = b * m + t / m + 1;
    R acc = 0;
    for (int e0 = first[slot]; e0 < first[slot + 1]; ++e0) {
      const int bl = src[e0];
      const int side = bl >> L;
      const int64_t kk = bl & ((int64_t(1) << L) - 1);
      int u, d;
      side_coords(side, n + 1, x, y, u, d);
      for (int e = 0; e < m; ++e) {
        // s1 = t_a - u with t_a = (k m + e)(n + 1)/n: exact integer numerator over n
        const int64_t num = (kk * m + e) * (int64_t)(n + 1) - (int64_t)u * n;
        const R qt = (R)qr[side * n + kk * m + e] * hR;
        acc += qt * seg_log_int<R>((R)num * invn, ell, (R)d);
      }
    }
    phib[((int64_t)rhs * nbnear + slot) * m * m + t] = acc;
  }
}

// ------------------------------------------------------------------ near field + L2P + sum
// One CTA per tile of TX x TY leaves, one thread per (leaf, row of m targets).  The
// weight image of the tile and its halo of R leaves, and the table of ln|d| over the
// stencil's node offsets, are staged in shared memory.  For every stencil row oy and
// source row sy a thread slides along the contiguous run of source leaves: per source
// leaf it loads the m weights of the row and the 2m-1 table values of the window and does
// m x m FMAs; partial sums are folded into Kahan-compensated accumulators (Sec. 7.1).
template <typename R>
struct P2PArgs {
  const R *wpad;
  const R *table;
  const cpx<R> *Lv;
  const R *phib;
  const int32_t *bslot;
  double *out;
  int n, npad, L, p, R_, Rn, HX, HY, TS, c0, tile_x, tile_y, nrhs;
  int64_t ncell, nbnear;
  int do_near, do_far, do_bnd;
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
__global__ void __launch_bounds__(256) k_p2p_final(P2PArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *halo = reinterpret_cast<R *>(smem_raw);
  R *tab = halo + (int64_t)A.HY * A.HX;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rhs = blockIdx.z;
  const int lx0 = blockIdx.x * A.tile_x, ly0 = blockIdx.y * A.tile_y;
  if (A.do_near) {
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
    const int tv = (2 * A.Rn + 1) * A.TS / VW;
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
  if (A.do_near) {
    const int Rr = A.R_;
    for (int oy = -Rr; oy <= Rr; ++oy) {
      const int ox0 = A.st.ox0[oy + Rr], ox1 = A.st.ox1[oy + Rr];
      if (ox0 > ox1) continue;
      for (int sy = 0; sy < M; ++sy) {
        const R *hrow = halo + ((lyl + Rr + oy) * M + sy) * A.HX + (lxl + Rr) * M;
        const R *trow = tab + (-oy * M + ty - sy + A.Rn) * A.TS + A.c0 + A.Rn - (M - 1);
        R part[M];
#pragma unroll
        for (int t = 0; t < M; ++t) part[t] = 0;
        for (int c = ox0; c <= ox1; ++c) {
          R w[M], tw[2 * M];
          lds_vec<R, M>(hrow + c * M, w);
          lds_vec<R, 2 * M>(trow - c * M, tw);
#pragma unroll
          for (int tx = 0; tx < M; ++tx)
#pragma unroll
            for (int sx = 0; sx < M; ++sx) part[tx] = fma(w[sx], tw[tx - sx + M - 1], part[tx]);
        }
#pragma unroll
        for (int t = 0; t < M; ++t) {  // Kahan
          const R y = part[t] - comp[t];
          const R s = sum[t] + y;
          comp[t] = (s - sum[t]) - y;
          sum[t] = s;
        }
      }
    }
  }
  const int gx = lx0 + lxl, gy = ly0 + lyl;
  const uint32_t leafc = morton_encode((uint32_t)gx, (uint32_t)gy);
  R far[M];
#pragma unroll
  for (int t = 0; t < M; ++t) far[t] = 0;
  if (A.do_far) {
    const cpx<R> *Lc = A.Lv + (int64_t)rhs * A.ncell * A.p + (level_offset(A.L) + leafc) * A.p;
    const R zy = (ty - R(0.5) * (M - 1)) / M;
    cpx<R> acc[M];
#pragma unroll
    for (int t = 0; t < M; ++t) acc[t] = mk<R>(0, 0);
    for (int k = A.p - 1; k >= 0; --k) {
      const cpx<R> Lk = Lc[k];
#pragma unroll
      for (int t = 0; t < M; ++t) acc[t] = acc[t] * mk<R>((t - R(0.5) * (M - 1)) / M, zy) + Lk;
    }
#pragma unroll
    for (int t = 0; t < M; ++t) far[t] = acc[t].re;
  }
  const R *pb = nullptr;
  if (A.do_bnd) {
    const int slot = A.bslot[leafc];
    if (slot >= 0) pb = A.phib + ((int64_t)rhs * A.nbnear + slot) * M * M + ty * M;
  }
  double *o = A.out + (int64_t)rhs * A.n * A.n + (int64_t)(gy * M + ty) * A.n + gx * M;
#pragma unroll
  for (int t = 0; t < M; ++t) {
    double v = ((double)sum[t] - (double)comp[t]) + (double)far[t];
    if (pb) v += (double)pb[t];
    o[t] = -v / (2.0 * PI);
  }
}

template <typename R, int M>
void launch_p2p(int L, const P2PArgs<R> &a, cudaStream_t s) {
  const int side = 1 << L;
  dim3 grid(side / a.tile_x, side / a.tile_y, a.nrhs);
  const int threads = a.tile_x * a.tile_y * M;
  const size_t smem = ((size_t)a.HY * a.HX + (size_t)(2 * a.Rn + 1) * a.TS) * sizeof(R);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    FMMPC_CUDA(cudaFuncSetAttribute(k_p2p_final<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    configured = smem;
  }
  k_p2p_final<R, M><<<grid, threads, smem, s>>>(a);
  FMMPC_LAUNCH_CHECK();
}

template <typename R, int P>
void launch_m2l_vol(fmmpc_handle &H, int nrhs, int with_bnd, cudaStream_t s) {
  const Geo &g = H.g;
  GeoDev gd{g.n, g.L, g.tnum, g.tden};
  k_m2l_vol<R, P><<<nblk(g.ncell * nrhs * 32), 256, 0, s>>>(
      gd, g.ncell, g.nbcell, nrhs, with_bnd, H.lists.m2l_first, H.lists.m2l_src, H.lists.vbv_first,
      H.lists.vbv_src, (const cpx<R> *)H.fb.Mv, (const cpx<R> *)H.fb.Mb, (cpx<R> *)H.fb.Lv);
  FMMPC_LAUNCH_CHECK();
}

template <typename R, int P>
void launch_m2l_bnd(fmmpc_handle &H, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  GeoDev gd{g.n, g.L, g.tnum, g.tden};
  k_m2l_bnd<R, P><<<nblk(g.nbcell * nrhs * 32), 256, 0, s>>>(
      gd, g.ncell, g.nbcell, nrhs, H.lists.vbb_first, H.lists.vbb_src, (const cpx<R> *)H.fb.Mv,
      (cpx<R> *)H.fb.Lb);
  FMMPC_LAUNCH_CHECK();
}

#define FMMPC_DISPATCH_P(p, CALL) \
  switch (p) {                     \
    case 4: CALL(4); break;        \
    case 6: CALL(6); break;        \
    case 8: CALL(8); break;        \
    case 10: CALL(10); break;      \
    case 12: CALL(12); break;      \
    case 16: CALL(16); break;      \
    default: throw Error(FMMPC_ERR_UNSUPPORTED, "expansion order p must be one of 4, 6, 8, 10, 12, 16"); \
  }

template <typename R>
void apply_impl(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  const Geo &g = H.g;
  const Lists &Ls = H.lists;
  cudaStream_t s = H.stream;
  R *wpad = (R *)H.fb.wpad;
  cpx<R> *Mv = (cpx<R> *)H.fb.Mv, *Lv = (cpx<R> *)H.fb.Lv;
  cpx<R> *Mb = (cpx<R> *)H.fb.Mb, *Lb = (cpx<R> *)H.fb.Lb;
  int64_t launches = 0;
  const int64_t N = (int64_t)g.n * g.n;
  // stage marks: event k opens stage k; a stage that does not run keeps stage_hit = false
  int cur = -1;
  auto mark = [&](int stage) {
    if (!H.timing) return;
    FMMPC_CUDA(cudaEventRecord(H.ev[stage], s));
    if (cur >= 0) H.stage_hit[cur] = true;
    cur = stage;
  };
  auto mark_end = [&]() {
    if (!H.timing) return;
    FMMPC_CUDA(cudaEventRecord(H.ev[fmmpc_handle::NSTAGE], s));
    if (cur >= 0) H.stage_hit[cur] = true;
  };
  if (H.timing)
    for (int k = 0; k < fmmpc_handle::NSTAGE; ++k) H.stage_hit[k] = false;
  mark(0);
  k_weights<R><<<nblk(N * nrhs), 256, 0, s>>>(g.n, g.npad, g.pad, g.h * g.h, N * nrhs, r, wpad);
  FMMPC_LAUNCH_CHECK();
  ++launches;
  const bool need_far = part != PART_NEAR;
  const bool with_bnd = part == PART_FULL || part == PART_VCOL || part == PART_Q;
  if (need_far) {
    mark(1);
    k_p2m_leaf<R><<<nblk(g.nleaf * nrhs * 32), 256, 0, s>>>(g, nrhs, wpad, Mv);
    FMMPC_LAUNCH_CHECK();
    ++launches;
    for (int l = g.L - 1; l >= 0; --l) {
      k_m2m_vol<R><<<nblk((int64_t(1) << (2 * l)) * nrhs, 128), 128, 0, s>>>(l, g.p, g.ncell, nrhs, Mv);
      FMMPC_LAUNCH_CHECK();
      ++launches;
    }
  }
  if (with_bnd) {
    mark(2);
#define CALL_MB(PP) launch_m2l_bnd<R, PP>(H, nrhs, s)
    FMMPC_DISPATCH_P(g.p, CALL_MB)
#undef CALL_MB
    k_root_const<R><<<1, 32, 0, s>>>(g.p, g.ncell, g.nbcell, nrhs, g.lnh, 0, Mv, Mb, Lv, Lb);
    launches += 2;
    for (int l = 0; l < g.L; ++l) {
      k_l2l_bnd<R><<<nblk(4 * (int64_t(1) << (l + 1)) * nrhs, 128), 128, 0, s>>>(l, g.n, g.p, g.nbcell, nrhs, Lb);
      ++launches;
    }
    k_colloc<R><<<nblk(g.nbleaf * nrhs * 32, 128), 128, 0, s>>>(g, nrhs, wpad, Lb, Ls.pvb_first, Ls.pvb_src, H.fb.vcol);
    FMMPC_LAUNCH_CHECK();
    ++launches;
    if (part == PART_VCOL) {
      FMMPC_CUDA(cudaMemcpyAsync(out, H.fb.vcol, sizeof(double) * g.NG * nrhs, cudaMemcpyDeviceToDevice, s));
      mark_end();
      H.launches = launches;
      return;
    }
    mark(3);
    k_bem_gemv<<<nblk((int64_t)g.NG * nrhs * 32), 256, 0, s>>>(g.NG, nrhs, H.Sinv, H.fb.vcol, H.fb.q);
    FMMPC_LAUNCH_CHECK();
    ++launches;
    if (part == PART_Q) {
      FMMPC_CUDA(cudaMemcpyAsync(out, H.fb.q, sizeof(double) * g.NG * nrhs, cudaMemcpyDeviceToDevice, s));
      mark_end();
      H.launches = launches;
      return;
    }
    mark(4);
    k_p2m_bnd<R><<<nblk(g.nbleaf * nrhs, 128), 128, 0, s>>>(g, nrhs, H.fb.q, Mb);
    FMMPC_LAUNCH_CHECK();
    ++launches;
    for (int l = g.L - 1; l >= 0; --l) {
      k_m2m_bnd<R><<<nblk(4 * (int64_t(1) << l) * nrhs, 128), 128, 0, s>>>(l, g.n, g.p, g.nbcell, nrhs, Mb);
      ++launches;
    }
    FMMPC_LAUNCH_CHECK();
  }
  if (need_far) {
    mark(5);
#define CALL_MV(PP) launch_m2l_vol<R, PP>(H, nrhs, with_bnd ? 1 : 0, s)
    FMMPC_DISPATCH_P(g.p, CALL_MV)
#undef CALL_MV
    k_root_const<R><<<1, 32, 0, s>>>(g.p, g.ncell, g.nbcell, nrhs, g.lnh, with_bnd ? 2 : 1, Mv, Mb, Lv, Lb);
    launches += 2;
    mark(6);
    for (int l = 0; l < g.L; ++l) {
      k_l2l_vol<R><<<nblk((int64_t(1) << (2 * (l + 1))) * nrhs, 128), 128, 0, s>>>(l, g.p, g.ncell, nrhs, Lv);
      ++launches;
    }
    FMMPC_LAUNCH_CHECK();
  }
  if (with_bnd && Ls.nbnear > 0) {
    mark(7);
    k_bnd_near<R><<<nblk(Ls.nbnear * nrhs * 32, 128), 128, 0, s>>>(g, Ls.nbnear, nrhs, Ls.pbv_leaf, Ls.pbv_first,
                                                                  Ls.pbv_src, H.fb.q, (R *)H.fb.phib);
    FMMPC_LAUNCH_CHECK();
    ++launches;
  }
  P2PArgs<R> a;
  a.wpad = wpad;
  a.table = (const R *)(part == PART_NEAR ? H.fb.table_lnh : H.fb.table);
  a.Lv = Lv;
  a.phib = (const R *)H.fb.phib;
  a.bslot = Ls.leaf_bslot;
  a.out = out;
  a.n = g.n; a.npad = g.npad; a.L = g.L; a.p = g.p; a.R_ = g.R; a.Rn = H.fb.Rn;
  a.HX = (H.tile_x + 2 * g.R) * g.m;
  a.HY = (H.tile_y + 2 * g.R) * g.m;
  a.TS = H.fb.table_stride; a.c0 = H.fb.table_c0;
  a.tile_x = H.tile_x; a.tile_y = H.tile_y; a.nrhs = nrhs;
  a.ncell = g.ncell; a.nbnear = Ls.nbnear;
  a.do_near = 1;
  a.do_far = need_far ? 1 : 0;
  a.do_bnd = (part == PART_FULL && Ls.nbnear > 0) ? 1 : 0;
  a.st = H.st;
  mark(8);
  switch (g.m) {
    case 4: launch_p2p<R, 4>(g.L, a, s); break;
    case 8: launch_p2p<R, 8>(g.L, a, s); break;
    case 16: launch_p2p<R, 16>(g.L, a, s); break;
    default: throw Error(FMMPC_ERR_UNSUPPORTED, "leaf side must be 4, 8 or 16");
  }
  ++launches;
  mark_end();
  H.launches = launches;
}

template <typename R>
void alloc_fmm(fmmpc_handle &H) {
  Geo &g = H.g;
  const int nr = H.nrhs_max;
  H.fb.wpad = H.pool.get<R>((size_t)nr * g.npad * g.npad);
  FMMPC_CUDA(cudaMemsetAsync(H.fb.wpad, 0, sizeof(R) * (size_t)nr * g.npad * g.npad, H.stream));
  H.fb.Mv = H.pool.get<cpx<R>>((size_t)nr * g.ncell * g.p);
  H.fb.Lv = H.pool.get<cpx<R>>((size_t)nr * g.ncell * g.p);
  H.fb.Mb = H.pool.get<cpx<R>>((size_t)nr * g.nbcell * g.p);
  H.fb.Lb = H.pool.get<cpx<R>>((size_t)nr * g.nbcell * g.p);
  H.fb.phib = H.pool.get<R>((size_t)nr * std::max<int64_t>(1, H.lists.nbnear) * g.m * g.m);
  H.fb.vcol = H.pool.get<double>((size_t)nr * g.NG);
  H.fb.q = H.pool.get<double>((size_t)nr * g.NG);
  // lattice table: rows dy in [-Rn, Rn], columns dx at c0 + Rn + dx; stride chosen so that
  // consecutive rows start 16 bytes apart modulo the 128-byte bank window
  const int Rn = g.R * g.m + g.m - 1;
  const int c0 = ((g.m - 1 - Rn) % 4 + 4) % 4;
  int TS = c0 + 2 * Rn + 2;
  while ((TS * (int)sizeof(R)) % 128 != 16) ++TS;
  H.fb.Rn = Rn;
  H.fb.table_c0 = c0;
  H.fb.table_stride = TS;
  H.fb.table_rows = 2 * Rn + 1;
  const double cself = -0.5 * std::log(2.0) - 1.5 + 0.25 * PI;  // mean of ln|x| on the unit cell
  std::vector<R> t0((size_t)(2 * Rn + 1) * TS, R(0)), t1((size_t)(2 * Rn + 1) * TS, R(0));
  for (int dy = -Rn; dy <= Rn; ++dy)
    for (int dx = -Rn; dx <= Rn; ++dx) {
      const double v = (dx == 0 && dy == 0) ? cself : 0.5 * std::log((double)dx * dx + (double)dy * dy);
      t0[(size_t)(dy + Rn) * TS + c0 + Rn + dx] = (R)v;
      t1[(size_t)(dy + Rn) * TS + c0 + Rn + dx] = (R)(v + g.lnh);
    }
  H.fb.table = H.pool.get<R>(t0.size());
  H.fb.table_lnh = H.pool.get<R>(t1.size());
  FMMPC_CUDA(cudaMemcpyAsync(H.fb.table, t0.data(), sizeof(R) * t0.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(H.fb.table_lnh, t1.data(), sizeof(R) * t1.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
}

}  // namespace

void init_fmm(fmmpc_handle &H) {
  double bin[MAXP + 1][MAXP + 1];
  for (int a = 0; a <= MAXP; ++a)
    for (int b = 0; b <= MAXP; ++b)
      bin[a][b] = (b == 0) ? 1.0 : (a == 0 ? 0.0 : bin[a - 1][b - 1] + bin[a - 1][b]);
  FMMPC_CUDA(cudaMemcpyToSymbol(c_binom, bin, sizeof(bin)));
  const int side = 1 << H.g.L;
  const int m = H.g.m;
  int tx = (m == 4) ? 8 : (m == 8 ? 8 : 4), ty = (m == 4) ? 8 : (m == 8 ? 4 : 4);
  H.tile_x = std::min(tx, side);
  H.tile_y = std::min(ty, side);
  if (H.prec == FMMPC_PREC_FP64) {
    if (m == 16) throw Error(FMMPC_ERR_UNSUPPORTED, "FP64 mode supports leaf side 4 or 8");
    alloc_fmm<double>(H);
  } else {
    alloc_fmm<float>(H);
  }
}

void apply_fmm(fmmpc_handle &H, int part, const double *r, double *out, int nrhs) {
  if (H.prec == FMMPC_PREC_FP64) apply_impl<double>(H, part, r, out, nrhs);
  else apply_impl<float>(H, part, r, out, nrhs);
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
  if (k >= (int64_t)(2 * Rn + 1) * TS) return;
  const int row = (int)(k / TS), col = (int)(k % TS);
  const int dy = row - Rn, dx = col - c0 - Rn;
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

// Device address of g_noalloc_scratch for the current device, resolved once per device.
cudaError_t noalloc_scratch(float **out) {
  static std::mutex mu;
  static float *ptr[NOALLOC_MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ptr[dev] = static_cast<float *>(p);
  }
  *out = ptr[dev];
  return cudaSuccess;
}

template <int M>
cudaError_t noalloc_launch(const P2PArgs<float> &a, int L, cudaStream_t s) {
  const int side = 1 << L;
  dim3 grid(side / a.tile_x, side / a.tile_y, 1);
  const size_t smem = ((size_t)a.HY * a.HX + (size_t)(2 * a.Rn + 1) * a.TS) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_p2p_final<float, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_p2p_final<float, M><<<grid, a.tile_x * a.tile_y * M, smem, s>>>(a);
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
  const int64_t tab_floats = (int64_t)(2 * Rn + 1) * TS;
  const int64_t need = tab_floats + (int64_t)npad * npad;
  if (need > NOALLOC_FLOATS)
    return set_global_error(FMMPC_ERR_INVALID, "near_field_noalloc: grid too large for the 16 MiB static scratch (n = 1024 with 8x8 leaves and theta 0.4 is the largest such grid)");
  float *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const double h = side / (n + 1);
  float *tab = scratch, *img = scratch + tab_floats;  // tab_floats is a multiple of 4: 16-byte aligned image
  k_noalloc_table<<<(unsigned)((tab_floats + 255) / 256), 256, 0, s>>>(tab, Rn, TS, c0, std::log(h));
  k_noalloc_image<<<(unsigned)(((int64_t)npad * npad + 255) / 256), 256, 0, s>>>(img, n, npad, pad, h * h, r_dev);
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  const int sidel = 1 << L;
  int tx = (m == 16) ? 4 : 8, ty = (m == 4) ? 8 : 4;
  tx = std::min(tx, sidel);
  ty = std::min(ty, sidel);
  P2PArgs<float> a{};
  a.wpad = img; a.table = tab; a.Lv = nullptr; a.phib = nullptr; a.bslot = nullptr; a.out = out_dev;
  a.n = n; a.npad = npad; a.L = L; a.p = 0; a.R_ = R; a.Rn = Rn;
  a.HX = (tx + 2 * R) * m; a.HY = (ty + 2 * R) * m; a.TS = TS; a.c0 = c0;
  a.tile_x = tx; a.tile_y = ty; a.nrhs = 1; a.ncell = 0; a.nbnear = 0;
  a.do_near = 1; a.do_far = 0; a.do_bnd = 0; a.st = st;
  switch (m) {
    case 4: e = noalloc_launch<4>(a, L, s); break;
    case 8: e = noalloc_launch<8>(a, L, s); break;
    default: e = noalloc_launch<16>(a, L, s); break;
  }
  if (e != cudaSuccess) return set_global_error(FMMPC_ERR_CUDA, cudaGetErrorString(e));
  return FMMPC_OK;
}

}  // namespace fmmpc
