// M2L (Sec. 5.3 item 3, the multipole-to-local translation) on the tensor cores, for the
// mixed-precision forms: TF32 or BF16 operands, FP32 accumulation.
//
// On the uniform quadtree the M2L list of a cell depends only on its position in its
// parent (the parity class c = (x & 1, y & 1)) and on which sources fall inside the domain,
// and in the scaled expansions (M~_k = M_k / rho^k, L~_n = L_n rho^n, offsets in cell units)
// the translation for offset o = t - s is a fixed complex p x p matrix C_o, the same at
// every level except for the ln rho term of L~_0:
//   C_o[0][0] = log o, C_o[0][k] = o^-k, C_o[n][0] = (-1)^(n+1) / (n o^n),
//   C_o[n][k] = (-1)^n (n+k-1)! / (n! (k-1)! o^(n+k)),  L~_0 += ln(rho) M~_0.
// Written as real 2p x 2p blocks, one level's M2L is a lattice convolution of the
// multipole image with fixed matrices.  The image of each level is split into its four
// parity sub-images, each zero-padded by 4 cells and flattened with row pitch P = S + 8
// (S = 2^(l-1) cells).  Target (i, j) of parity class c = (cx, cy) and offset o take source
// 2 (i, j) + c - o, which lies in sub-image ((cx - ox) & 1, (cy - oy) & 1) at (i + dx, j + dy)
// with (dx, dy) = floor((c - o) / 2): the same target position in all four classes reads
// the same source row for a shift (source parity, dx, dy), each class through its own
// offset.  So one CTA takes 128 consecutive flattened target positions (M = 128) of all
// four classes and sweeps the 124 shifts, D[t][W c + u] += sum_v X[t + dy P + dx][v] B_s[W c + u][v],
// with the four classes' matrices stacked along N = 4 W (zero rows where a class has no
// offset for the shift), K = the multipole inputs.  Per class the W outputs (W = 24 for
// p <= 11, else 32) are the 2p real parts of L~ and, in outputs W - 2 and W - 1, the two
// sums of M~_0 that carry ln rho.
// Padding targets are computed and dropped.  The low-order terms dominate the translated
// field and meet the large log o + ln rho, so their products are split hi + lo in the
// spare K columns (K = 32 for TF32: M~_0..2 at p = 10; K = 48 for BF16: M~_0..6): rounded
// input x rounded matrix, input residual x rounded matrix, rounded input x matrix residual.
//
// Operands use the 128-byte swizzle (one 128-byte row per cell), so a shifted window is a
// descriptor offset.  Shifts are grouped by (source parity, dy); one 144-row window of the
// source sub-image serves every dx of a group.  Warp 0 streams the windows and warp 10 the
// B blocks of each group (one bulk copy per group), each through its own ring; warp 1
// issues the MMAs, one fresh 128-column TMEM accumulator per group (four in flight), and
// warps 2-9 add each into FP32 sums: one long chain of MMAs would drift with the tensor
// core's truncating adds (~2^-24 of the partial per MMA).  When a level has too few tiles to fill the GPU, each tile's groups are split
// into two parts run by two CTAs, which add into zeroed L~.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>

#include <cuda_bf16.h>

#include "handle.cuh"
#include "tc.cuh"

namespace fmmpc {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

constexpr int M2L_WROWS = 144;                  // window rows (128 targets + 2 x 4 shift + alignment)
constexpr int M2L_WBYTES = M2L_WROWS * 128;     // 18 KB
constexpr int M2L_NWIN = 3;                     // window slots
constexpr int M2L_NACC = 4;                     // TMEM accumulators in flight (128-column stride)
constexpr int M2L_NGR = 16;                     // group barriers (> B slots, > M2L_NACC)
constexpr int M2L_EPI_WARPS = 8;
constexpr int M2L_THREADS = 96 + 32 * M2L_EPI_WARPS;  // window producer, MMA, epilogue, B producer
constexpr int M2L_TAIL = 256;                   // zero rows after each sub-image (window overrun)
constexpr int M2L_MAXGRP = 64, M2L_MAXSH = 255;  // per part: (source parity, dy) groups, shifts
// W outputs per class (2p real parts of L~, the two M~_0 sums in the last two): N = 4 W;
// one shift's B block is N rows of 128 bytes; as many B slots as fit beside the windows
template <int W>
struct M2lShape {
  static constexpr int N = 4 * W;
  static constexpr int BBYTES = N * 128;
  static constexpr int NB = W == 24 ? 13 : 10;
  static constexpr int SMEM = M2L_NWIN * M2L_WBYTES + NB * BBYTES + 1024;
};

struct M2lArgs {
  const unsigned char *img;     // [nrhs][rows_per_rhs][128 B]
  const unsigned char *bmat;    // [shift][4 W][128 B]
  const int2 *tiles;            // (level, f0)
  const int4 *groups;           // (source parity, dy, first shift, count), by (source parity, dy)
  const int *dxs;               // [shift]: dx of the shift
  cpx<float> *Lv;               // [nrhs][ncell][p]
  int *err;
  int64_t rows_per_rhs, ncell;
  int64_t lev_row0[24];         // first image row of level l (parity 0)
  int lev_P[24];
  int gpart[3], gpart_sh[3];    // groups and shifts of each part
  int p, n, nks, nsplit, nparts, sbase;
};

__device__ __forceinline__ int floor8(int x) { return x & ~7; }

template <int KIND>
__device__ __forceinline__ float m2l_round(float x) {
  if (KIND == 0) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  return __bfloat162float(__float2bfloat16_rn(x));
}

// K input v of a cell: v < 2p the rounded real parts of M~ (Re M~_0, Im M~_0, Re M~_1, ...);
// for j < nsplit, v = sb + 4j + {0, 1}: the rounding residual of M~_j (meets B's rounded
// column j), v = sb + 4j + {2, 3}: the rounded M~_j again (meets the residual of column j).
// sb (split base) is 2p.
template <int KIND>
__device__ __forceinline__ float m2l_input(const cpx<float> *M, int v, int p, int nsplit, int sb) {
  if (v < 2 * p) {
    const float x = (v & 1) ? M[v >> 1].im : M[v >> 1].re;
    return m2l_round<KIND>(x);
  }
  if (v < sb) return 0.f;
  const int w = v - sb, j = w >> 2, e = w & 3;
  if (j >= nsplit) return 0.f;
  const float x = (e & 1) ? M[j].im : M[j].re;
  const float hi = m2l_round<KIND>(x);
  return e < 2 ? m2l_round<KIND>(x - hi) : hi;
}

// Multipole image rows: thread per (rhs, cell at level >= 2, 16-byte chunk).  Also clears
// the local expansions of levels 0 and 1, which have no M2L sources, and those of every
// level when the M2L is split into parts that add.
template <int KIND>
__global__ void k_m2l_pack(M2lArgs a, int nrhs, int64_t ncell_lo, int64_t ncell_hi, const cpx<float> *__restrict__ Mv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (ncell_hi - ncell_lo) * 8;
  if (t < (int64_t)nrhs * level_offset(2) * a.p) {
    const int64_t rhs = t / (level_offset(2) * a.p), k = t % (level_offset(2) * a.p);
    a.Lv[rhs * a.ncell * a.p + k] = mk<float>(0.f, 0.f);
  }
  if (t >= (int64_t)nrhs * per) return;
  const int64_t rhs = t / per, rem = t % per;
  const int64_t gidx = ncell_lo + rem / 8;
  const int chunk = (int)(rem % 8);
  int l = 2;
  while (level_offset(l + 1) <= gidx) ++l;
  int x, y;
  morton_decode((uint32_t)(gidx - level_offset(l)), x, y);
  const int P = a.lev_P[l];
  const int q = (x & 1) + 2 * (y & 1);
  const int64_t f = (int64_t)((y >> 1) + 4) * P + (x >> 1) + 4;
  const int64_t row = rhs * a.rows_per_rhs + a.lev_row0[l] + (int64_t)q * ((int64_t)P * P + M2L_TAIL) + f;
  const cpx<float> *M = Mv + (rhs * a.ncell + gidx) * a.p;
  if (a.nparts > 1) {  // the M2L parts add into L~
    cpx<float> *Lc = a.Lv + (rhs * a.ncell + gidx) * a.p;
    if (chunk < a.p) Lc[chunk] = mk<float>(0.f, 0.f);
    if (chunk + 8 < a.p) Lc[chunk + 8] = mk<float>(0.f, 0.f);
  }
  uint32_t w[4];
  if (KIND == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = __float_as_uint(m2l_input<KIND>(M, 4 * chunk + e, a.p, a.nsplit, a.sbase));
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 b0 = __float2bfloat16_rn(m2l_input<KIND>(M, 8 * chunk + 2 * e, a.p, a.nsplit, a.sbase));
      const __nv_bfloat16 b1 = __float2bfloat16_rn(m2l_input<KIND>(M, 8 * chunk + 2 * e + 1, a.p, a.nsplit, a.sbase));
      w[e] = (uint32_t)*reinterpret_cast<const uint16_t *>(&b0) | ((uint32_t)*reinterpret_cast<const uint16_t *>(&b1) << 16);
    }
  }
  uint4 *dst = reinterpret_cast<uint4 *>(const_cast<unsigned char *>(a.img) + row * 128) + (chunk ^ (int)(f & 7));
  *dst = make_uint4(w[0], w[1], w[2], w[3]);
}

// L~ of target (i, j) of class c at level l from its W outputs t[0 .. W): 2p real parts,
// and in the last two the sums of Re M~_0 and Im M~_0 that carry the ln rho term of L~_0.
template <int W>
__device__ __forceinline__ void m2l_store(const M2lArgs &a, const float *t, int l, int c, int i, int j, int rhs,
                                          float lnrho) {
  const int x = 2 * i + (c & 1), y = 2 * j + (c >> 1);
  const int64_t gidx = level_offset(l) + morton_encode((uint32_t)x, (uint32_t)y);
  cpx<float> *L = a.Lv + ((int64_t)rhs * a.ncell + gidx) * a.p;
  const float l0r = t[0] + lnrho * t[W - 2], l0i = t[1] + lnrho * t[W - 1];
  if (a.nparts == 1) {
    L[0] = mk<float>(l0r, l0i);
#pragma unroll
    for (int nn = 1; nn < W / 2 - 1; ++nn)
      if (nn < a.p) L[nn] = mk<float>(t[2 * nn], t[2 * nn + 1]);
  } else {
    // two parts add onto zeros: (0 + a) + b = (0 + b) + a, so the order of the two atomic
    // adds does not change the result
    float2 *L2 = reinterpret_cast<float2 *>(L);
    atomicAdd(L2, make_float2(l0r, l0i));
#pragma unroll
    for (int nn = 1; nn < W / 2 - 1; ++nn)
      if (nn < a.p) atomicAdd(L2 + nn, make_float2(t[2 * nn], t[2 * nn + 1]));
  }
}

template <int KIND, int W>
__global__ void __launch_bounds__(M2L_THREADS, 1) k_m2l_tc(M2lArgs a) {
  using SH = M2lShape<W>;
  constexpr int N = SH::N, NB = SH::NB, BBYTES = SH::BBYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // wfull: a window landed; bfull (ring of M2L_NGR groups): a group's B blocks landed;
  // gdone (same ring): the group's MMAs completed (one commit), which frees its window slot,
  // its B slots and its accumulator
  __shared__ uint64_t wfull[M2L_NWIN], bfull[M2L_NGR], gdone[M2L_NGR], acc_empty[M2L_NACC], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, w_used, b_used;
  // this part's groups and shifts in this CTA's order, off the issue path
  __shared__ int4 sgrp[M2L_MAXGRP];           // (source parity, dy, first local shift, count)
  __shared__ unsigned char sdx_b[M2L_MAXSH];  // dx + 4 of each local shift (0 .. 8)
  __shared__ unsigned char sgof[M2L_MAXSH];   // local group of each local shift
  __shared__ short sbi[M2L_MAXSH];            // B block (shift index) of each local shift
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char *wbuf = smem, *bbuf = smem + M2L_NWIN * M2L_WBYTES;
  const int2 tile = a.tiles[blockIdx.x];
  const int l = tile.x, f0 = tile.y, part = blockIdx.y, rhs = blockIdx.z;
  const int P = a.lev_P[l];
  const int g0 = a.gpart[part], ng = a.gpart[part + 1] - g0;
  const int sh0 = a.gpart_sh[part], nsh = a.gpart_sh[part + 1] - sh0;
  // Every CTA sweeps the same shifts; started in step they would all read the same B block
  // from the same few L2 slices at the same time.  Each tile therefore starts its sweep at
  // group (tile mod ng) and wraps around.  The order of the sums is then fixed per tile and
  // the same for every right-hand side.
  const int rot = (int)(blockIdx.x % (unsigned)max(ng, 1));
  const int shr = ng > 0 ? a.groups[g0 + rot].z : sh0;  // first shift of the sweep
  for (int j = tid; j < ng; j += blockDim.x) {
    const int o = j + rot < ng ? j + rot : j + rot - ng;
    const int4 g = a.groups[g0 + o];
    const int st = g.z >= shr ? g.z - shr : g.z - sh0 + (sh0 + nsh - shr);  // first local shift
    sgrp[j] = make_int4(g.x, g.y, st, g.w);
    for (int k = 0; k < g.w; ++k) {
      sgof[st + k] = (unsigned char)j;
      sdx_b[st + k] = (unsigned char)(a.dxs[g.z + k] + 4);
      sbi[st + k] = (short)(g.z + k);
    }
  }
  if (tid == 0) {
    for (int s = 0; s < M2L_NWIN; ++s) tc::mbar_init(&wfull[s], 1);
    for (int s = 0; s < M2L_NGR; ++s) tc::mbar_init(&bfull[s], 1);
    for (int s = 0; s < M2L_NGR; ++s) tc::mbar_init(&gdone[s], 1);
    for (int b = 0; b < M2L_NACC; ++b) tc::mbar_init(&acc_empty[b], M2L_EPI_WARPS);
    tc::mbar_init(&done, 1);
    tc::mbar_init_fence();
    abort_flag = 0;
    w_used = b_used = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, 128 * M2L_NACC);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  int w_issued = 0, b_issued = 0;
  // window slot gi % M2L_NWIN is free once group gi - M2L_NWIN is done, B slot b % NB once
  // the group holding shift b - NB is done; groups complete in order.  Each producer keeps
  // the highest group it has seen done.
  int known = -1;
  auto wait_done = [&](int gq) -> bool {
    if (gq <= known) return true;
    if (!tc::mbar_wait(&gdone[gq % M2L_NGR], (gq / M2L_NGR) & 1, &abort_flag)) return false;
    known = gq;
    return true;
  };
  if (warp == 0) {
    if (lane == 0) {
      // window producer: per group its 144-row source window
      bool ok = true;
      for (int gi = 0; gi < ng && !abort_flag; ++gi) {
        const int4 g = sgrp[gi];  // (source parity, dy, first local shift, count)
        if (!wait_done(gi - M2L_NWIN)) { ok = false; break; }
        const int w0 = floor8(f0 + g.y * P - 4);
        const unsigned char *src = a.img + ((int64_t)rhs * a.rows_per_rhs + a.lev_row0[l] +
                                            (int64_t)g.x * ((int64_t)P * P + M2L_TAIL) + w0) * 128;
        const int ws = gi % M2L_NWIN;
        tc::mbar_expect_tx(&wfull[ws], M2L_WBYTES);
        tc::bulk_g2s(wbuf + ws * M2L_WBYTES, src, M2L_WBYTES, &wfull[ws]);
        w_issued = gi + 1;
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
    }
  } else if (warp == 1 + M2L_EPI_WARPS + 1) {
    if (lane == 0) {
      // B producer: per group the B blocks of its shifts (each the four classes' translation
      // matrices stacked along N) in one bulk copy, two where the ring of NB shift slots
      // wraps.  A bulk copy costs about the same time whatever its size up to ~50 KB and an
      // SM runs them one after another, so one copy per group instead of one per shift.
      // The group's shifts are consecutive B blocks and consecutive local shifts, and slot
      // b % NB was last used by shift b - NB: the group of the group's last shift minus NB
      // must be done.  That group is at most NB groups back, so the previous phase of this
      // group's barrier (M2L_NGR > NB groups back) has completed.
      bool ok = true;
      for (int gi = 0; gi < ng && !abort_flag; ++gi) {
        const int4 g = sgrp[gi];
        const int blast = g.z + g.w - 1;
        if (blast >= NB && !wait_done(sgof[blast - NB])) { ok = false; break; }
        const int s0 = g.z % NB, n1 = min(g.w, NB - s0);
        uint64_t *bar = &bfull[gi % M2L_NGR];
        const unsigned char *src = a.bmat + (int64_t)sbi[g.z] * BBYTES;
        tc::mbar_expect_tx(bar, (uint32_t)(g.w * BBYTES));
        tc::bulk_g2s(bbuf + s0 * BBYTES, src, (uint32_t)(n1 * BBYTES), bar);
        if (n1 < g.w) tc::bulk_g2s(bbuf, src + (int64_t)n1 * BBYTES, (uint32_t)((g.w - n1) * BBYTES), bar);
        b_issued = gi + 1;
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: per group one fresh accumulator and one commit; per shift M = 128
      // targets, N = 4 classes x W outputs
      const uint32_t idesc = KIND == 0 ? tc::idesc_tf32(128, N)
                                       : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                          ((128u >> 4) << 24));
      const int nks = a.nks;  // 1-4 K steps of 32 bytes (8 TF32 or 16 BF16 inputs each)
      // descriptor low words of window slot 0 and B slot 0 (+8 per 128-byte row, +2 per K step)
      const uint32_t wlo0 = tc::desc_lo(tc::smem_addr(wbuf)), blo0 = tc::desc_lo(tc::smem_addr(bbuf));
      bool ok = true;
      int bs = 0;  // B slot of the current shift (local shifts run 0, 1, ... across the groups)
      for (int gi = 0; gi < ng && ok; ++gi) {
        const int ab = gi % M2L_NACC, ws = gi % M2L_NWIN;
        if (!tc::mbar_wait(&wfull[ws], (gi / M2L_NWIN) & 1, &abort_flag)) { ok = false; break; }
        w_used = gi + 1;
        if (gi >= M2L_NACC && !tc::mbar_wait(&acc_empty[ab], ((gi / M2L_NACC) - 1) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        if (!tc::mbar_wait(&bfull[gi % M2L_NGR], (gi / M2L_NGR) & 1, &abort_flag)) { ok = false; break; }
        b_used = gi + 1;
        tc::fence_after();
        const int4 g = sgrp[gi];
        const int w0 = floor8(f0 + g.y * P - 4);
        // first row of shift dx in the window: (f0 + dy P - w0 - 4) + (dx + 4), both terms >= 0
        const uint32_t alo_g = wlo0 + (uint32_t)(ws * (M2L_WBYTES >> 4) + (f0 + g.y * P - w0 - 4) * 8);
        const unsigned char *gdx = sdx_b + g.z;
        const uint32_t d = tmem + 128 * ab;
        for (int k = 0; k < g.w; ++k) {
          const uint32_t alo = alo_g + 8u * gdx[k], blo = blo0 + (uint32_t)bs * (BBYTES >> 4);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            if (ks < nks) {
              const uint64_t ad = tc::desc_of(alo + 2 * ks), bd = tc::desc_of(blo + 2 * ks);
              const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
              if (KIND == 0) {
                tc::mma_tf32(d, ad, bd, idesc, acc);
              } else {
                tc::mma_f16(d, ad, bd, idesc, acc);
              }
            }
          }
          if (++bs == NB) bs = 0;
        }
        tc::commit(&gdone[gi % M2L_NGR]);
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
      tc::commit(&done);
    }
  } else if (warp <= 1 + M2L_EPI_WARPS) {
    // epilogue: warps 2-9; warp w reads TMEM lanes 32 (w % 4) .. + 31 (one target each) and
    // the 2W columns of classes 2h, 2h + 1, h = (w - 2) / 4, in loads of 16 columns; each
    // group's accumulator is added into plain FP32 sums (a group is at most a few dozen
    // MMAs, so the tensor core's truncating adds stay near 2^-24 relative)
    const int qd = warp & 3, h = (warp - 2) >> 2;
    float sum[2 * W];
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) sum[i] = 0.0f;
    bool ok = true;
    for (int gi = 0; gi < ng; ++gi) {
      const int ab = gi % M2L_NACC;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&gdone[gi % M2L_NGR], (gi / M2L_NGR) & 1, &abort_flag))) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + 128 * ab + 2 * W * h;
#pragma unroll
      for (int q = 0; q < 2 * W / 16; ++q) {
        float v[16];
        tc::tmem_ld16(ta + 16 * q, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[ab]);
    }
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicOr(a.err, 2);
    }
    const int f = f0 + 32 * qd + lane;
    const int S = P - 8;
    const int i = f % P - 4, j = f / P - 4;
    if (ok && !abort_flag && i >= 0 && i < S && j >= 0 && j < S) {
      const float lnrho = logf((float)(a.n >> l));
      m2l_store<W>(a, sum, l, 2 * h, i, j, rhs, lnrho);
      m2l_store<W>(a, sum + W, l, 2 * h + 1, i, j, rhs, lnrho);
    }
  }
  __syncwarp();
  const bool finished = __all_sync(0xffffffffu, tc::mbar_wait(&done, 0, nullptr));  // warp-uniform
  if (!finished && lane == 0) atomicOr(a.err, 4);
  tc::fence_before();
  __syncthreads();
  if (abort_flag && lane == 0) {  // copies still in flight land before the block exits
    if (warp == 0)
      for (int u = w_used; u < w_issued; ++u) tc::mbar_wait(&wfull[u % M2L_NWIN], (u / M2L_NWIN) & 1, nullptr);
    if (warp == 1 + M2L_EPI_WARPS + 1)
      for (int u = b_used; u < b_issued; ++u) tc::mbar_wait(&bfull[u % M2L_NGR], (u / M2L_NGR) & 1, nullptr);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 128 * M2L_NACC);
  }
}

// Offsets of the M2L lists by target parity class (levels >= 2): table[c][(oy+7)*15 + ox+7].
__global__ void k_m2l_offsets(int L, const int32_t *__restrict__ first, const int32_t *__restrict__ src,
                              int *__restrict__ table, int *__restrict__ err) {
  const int64_t gidx = level_offset(2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= level_offset(L + 1)) return;
  int l = 2;
  while (level_offset(l + 1) <= gidx) ++l;
  int tx, ty;
  morton_decode((uint32_t)(gidx - level_offset(l)), tx, ty);
  const int c = (tx & 1) + 2 * (ty & 1);
  for (int e = first[gidx]; e < first[gidx + 1]; ++e) {
    int sx, sy;
    morton_decode((uint32_t)src[e], sx, sy);
    const int ox = tx - sx, oy = ty - sy;
    if (ox < -7 || ox > 7 || oy < -7 || oy > 7) {
      atomicOr(err, 1);
      continue;
    }
    table[c * 225 + (oy + 7) * 15 + ox + 7] = 1;
  }
}

// Every list must be exactly its class's offsets with an in-domain source.
__global__ void k_m2l_verify(int L, const int32_t *__restrict__ first, const int *__restrict__ table,
                             int *__restrict__ err) {
  const int64_t gidx = level_offset(2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= level_offset(L + 1)) return;
  int l = 2;
  while (level_offset(l + 1) <= gidx) ++l;
  int tx, ty;
  morton_decode((uint32_t)(gidx - level_offset(l)), tx, ty);
  const int c = (tx & 1) + 2 * (ty & 1), NL = 1 << l;
  int expect = 0;
  for (int oy = -7; oy <= 7; ++oy)
    for (int ox = -7; ox <= 7; ++ox)
      if (table[c * 225 + (oy + 7) * 15 + ox + 7]) {
        const int sx = tx - ox, sy = ty - oy;
        if (sx >= 0 && sx < NL && sy >= 0 && sy < NL) ++expect;
      }
  if (expect != first[gidx + 1] - first[gidx]) atomicOr(err, 2);
}

float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

uint16_t bf16_round_host(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);  // nearest, ties to even
  return (uint16_t)(u >> 16);
}

float tf32_round_host_m2l(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x1000u;
    u &= 0xffffe000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

bool tc_m2l_eligible(const fmmpc_handle &H) {
  // W <= 32 outputs per class hold 2p + 2; K (32 TF32 or BF16 inputs per 128-byte row) holds 2p
  return (H.prec == FMMPC_PREC_MIXED_BF16 || H.prec == FMMPC_PREC_MIXED_TF32) && H.g.L >= 2 && 2 * H.g.p + 2 <= 32;
}

void init_tc_m2l(fmmpc_handle &H, DevPool &tmp) {
  TcM2L &T = H.tcm;
  T.enabled = false;
  if (!tc_m2l_eligible(H)) return;
  const Geo &g = H.g;
  const int L = g.L, p = g.p;
  T.kind = (H.prec == FMMPC_PREC_MIXED_TF32) ? 0 : 1;
  T.width = (2 * p + 2 <= 24) ? 24 : 32;  // outputs per class
  // hi/lo splits of the leading multipoles in the spare K columns: TF32 32 inputs (4 K steps
  // of 8, one 128-byte row), BF16 48 (3 K steps of 16).  A BF16 hi + lo pair carries about
  // 16 bits, so the BF16 products stay near 2^-16 relative however many terms are split
  // (splitting every term, or moving the corrections to K steps of their own, measured the
  // same z error, 4.5e-5 at 1024^2): three K steps are the cheapest at that accuracy.
  const int kcap = T.kind == 0 ? 32 : 48;
  T.sbase = 2 * p;
  T.nsplit = std::max(0, std::min(p, (kcap - T.sbase) / 4));
  // offset sets by class, from the lists themselves, then checked against every list
  int *dtab = tmp.get<int>(4 * 225), *derr = tmp.get<int>(1);
  FMMPC_CUDA(cudaMemsetAsync(dtab, 0, sizeof(int) * 4 * 225, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), H.stream));
  const int64_t nt = level_offset(L + 1) - level_offset(2);
  k_m2l_offsets<<<nblk(nt), 256, 0, H.stream>>>(L, H.lists.m2l_first, H.lists.m2l_src, dtab, derr);
  k_m2l_verify<<<nblk(nt), 256, 0, H.stream>>>(L, H.lists.m2l_first, dtab, derr);
  FMMPC_LAUNCH_CHECK();
  std::vector<int> tab(4 * 225);
  int herr = 0;
  FMMPC_CUDA(cudaMemcpyAsync(tab.data(), dtab, sizeof(int) * 4 * 225, cudaMemcpyDeviceToHost, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, H.stream));
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
  if (herr) throw Error(FMMPC_ERR_INVALID, "tensor-core M2L: the M2L lists are not translation invariant");
  // shifts (source parity, dy, dx) with the offset each class translates over it, grouped
  // by (source parity, dy) and sorted by dx: target (i, j) of class c = (cx, cy) takes
  // source cell 2 (i, j) + (cx, cy) - o, which sits in source parity sub-image
  // ((cx - ox) & 1, (cy - oy) & 1) at (i + dx, j + dy), dx = floor((cx - ox) / 2)
  std::map<std::pair<int, int>, std::map<int, std::array<int, 4>>> bykey;  // (sp, dy) -> dx -> offset per class
  for (int c = 0; c < 4; ++c) {
    const int cx = c & 1, cy = c >> 1;
    for (int oy = -7; oy <= 7; ++oy)
      for (int ox = -7; ox <= 7; ++ox) {
        if (!tab[c * 225 + (oy + 7) * 15 + ox + 7]) continue;
        const int spx = (cx - ox) & 1, spy = (cy - oy) & 1;
        const int dx = (cx - ox - spx) / 2, dy = (cy - oy - spy) / 2;
        auto &row = bykey[{spx + 2 * spy, dy}];
        if (!row.count(dx)) row[dx] = {-1, -1, -1, -1};
        row[dx][c] = (oy + 7) * 15 + ox + 7;
      }
  }
  std::vector<int4> groups;
  std::vector<int> dxs;
  std::vector<std::array<int, 4>> shift_ofs;
  for (auto &kv : bykey) {
    groups.push_back(make_int4(kv.first.first, kv.first.second, (int)dxs.size(), (int)kv.second.size()));
    for (auto &e : kv.second) {
      dxs.push_back(e.first);
      shift_ofs.push_back(e.second);
    }
  }
  const int nshift = (int)dxs.size(), ngrp = (int)groups.size();
  // the 144-row window holds the 128 targets shifted by dx in [-4, 4]
  for (int dx : dxs)
    if (dx < -4 || dx > 4) throw Error(FMMPC_ERR_UNSUPPORTED, "tensor-core M2L: shift outside the source window");
  // images and tiles (128 consecutive flattened targets of one level, all four classes)
  int64_t rows = 0;
  std::vector<int2> tiles;
  for (int l = 0; l < 24; ++l) {
    T.lev_row0[l] = 0;
    T.lev_P[l] = 0;
  }
  for (int l = 2; l <= L; ++l) {
    const int S = 1 << (l - 1), P = S + 8;
    T.lev_P[l] = P;
    T.lev_row0[l] = rows;
    rows += 4 * ((int64_t)P * P + M2L_TAIL);
    const int fs = 4 * P + 4, fe = (S + 3) * P + S + 3;
    for (int f0 = fs; f0 <= fe; f0 += 128) tiles.push_back(make_int2(l, f0));
  }
  T.rows_per_rhs = rows;
  T.ntiles = (int)tiles.size();
  // with few tiles per right-hand side, each tile's groups are split into two parts of about
  // equal shift counts (two CTAs); the choice depends on the geometry only, so a batch and
  // its single right-hand sides take the same sums
  int nsm = 0;
  FMMPC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
  T.nparts = (2 * T.ntiles <= nsm && ngrp >= 2) ? 2 : 1;
  T.gpart[0] = 0;
  T.gpart[T.nparts] = ngrp;
  if (T.nparts == 2) {
    int best = 1, bestd = 1 << 30;
    for (int k = 1; k < ngrp; ++k) {
      const int d = std::abs(2 * groups[k].z - nshift);
      if (d < bestd) bestd = d, best = k;
    }
    T.gpart[1] = best;
  }
  for (int q = 0; q <= T.nparts; ++q) T.gpart_sh[q] = T.gpart[q] < ngrp ? groups[T.gpart[q]].z : nshift;
  int maxcnt = 0;
  for (auto &gr : groups) maxcnt = std::max(maxcnt, gr.w);
  for (int q = 0; q < T.nparts; ++q)
    if (T.gpart[q + 1] - T.gpart[q] > M2L_MAXGRP || T.gpart_sh[q + 1] - T.gpart_sh[q] > M2L_MAXSH ||
        maxcnt > (T.width == 24 ? M2lShape<24>::NB : M2lShape<32>::NB))
      throw Error(FMMPC_ERR_UNSUPPORTED, "tensor-core M2L: too many shifts");
  T.nofs_total = nshift;
  // B operands, one 4W x 128-byte block per shift: row W c + u is output u of class c
  // (2p real parts of L~; in W - 2, W - 1 the sums of Re M~_0 and Im M~_0), zero where class c has no
  // offset for the shift; column v is input v of the multipole image row
  const int W = T.width, bbytes = 4 * W * 128;
  std::vector<unsigned char> B((size_t)nshift * bbytes, 0);
  std::vector<double> fact(2 * p + 2, 1.0);
  for (int i = 1; i < (int)fact.size(); ++i) fact[i] = fact[i - 1] * i;
  for (int q = 0; q < nshift; ++q)
    for (int c = 0; c < 4; ++c) {
      const int oi = shift_ofs[q][c];
      if (oi < 0) continue;
      const std::complex<double> o((double)(oi % 15 - 7), (double)(oi / 15 - 7));
      std::vector<std::complex<double>> C((size_t)p * p);
      for (int nn = 0; nn < p; ++nn)
        for (int k = 0; k < p; ++k) {
          std::complex<double> cv;
          if (nn == 0 && k == 0) cv = std::log(o);
          else if (nn == 0) cv = 1.0 / std::pow(o, k);
          else if (k == 0) cv = ((nn % 2) ? 1.0 : -1.0) / ((double)nn * std::pow(o, nn));
          else cv = ((nn % 2) ? -1.0 : 1.0) * fact[nn + k - 1] / (fact[nn] * fact[k - 1]) / std::pow(o, nn + k);
          C[(size_t)nn * p + k] = cv;
        }
      auto Breal = [&](int u, int v) -> double {  // real form of C_o, plus the two M~_0 sum rows
        if (u >= W - 2) return (u - (W - 2) == v) ? 1.0 : 0.0;
        const std::complex<double> cv = C[(size_t)(u / 2) * p + v / 2];
        if ((u & 1) == 0) return (v & 1) ? -cv.imag() : cv.real();
        return (v & 1) ? cv.real() : cv.imag();
      };
      auto put = [&](int u, int v, double val) {
        const int n = W * c + u;
        unsigned char *row = B.data() + (size_t)q * bbytes + (size_t)n * 128;
        if (T.kind == 0) {
          const int ch = v / 4, e = v % 4;
          const float f = tf32_round_host_m2l(val);
          std::memcpy(row + ((ch ^ (n & 7)) * 16) + 4 * e, &f, 4);
        } else {
          const int ch = v / 8, e = v % 8;
          const uint16_t b = bf16_round_host(val);
          std::memcpy(row + ((ch ^ (n & 7)) * 16) + 2 * e, &b, 2);
        }
      };
      std::vector<int> outs;  // 2p real parts of L~, the two M~_0 sums in outputs W - 2, W - 1
      for (int u = 0; u < 2 * p; ++u) outs.push_back(u);
      outs.push_back(W - 2);
      outs.push_back(W - 1);
      for (int u : outs)
        for (int v = 0; v < 2 * p; ++v) put(u, v, Breal(u, v));
      // split columns: residual inputs meet the rounded column, rounded inputs the column residual
      for (int j = 0; j < T.nsplit; ++j)
        for (int u : outs)
          for (int e = 0; e < 2; ++e) {
            const double full = Breal(u, 2 * j + e);
            const double hi = T.kind == 0 ? (double)tf32_round_host_m2l(full) : bf16_value(bf16_round_host(full));
            put(u, T.sbase + 4 * j + e, full);
            put(u, T.sbase + 4 * j + 2 + e, full - hi);
          }
    }
  T.smem = W == 24 ? M2lShape<24>::SMEM : M2lShape<32>::SMEM;
  int maxsm = 0;
  FMMPC_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0));
  if (T.smem + 8192 > maxsm) throw Error(FMMPC_ERR_UNSUPPORTED, "tensor-core M2L: not enough shared memory");
  T.img = H.pool.get<unsigned char>((size_t)H.nrhs_max * rows * 128);
  FMMPC_CUDA(cudaMemsetAsync(T.img, 0, (size_t)H.nrhs_max * rows * 128, H.stream));
  T.bmat = H.pool.get<unsigned char>(B.size());
  T.tiles = H.pool.get<int2>(tiles.size());
  T.groups = H.pool.get<int4>(groups.size());
  T.dxs = H.pool.get<int>(dxs.size());
  T.err = H.pool.get<int>(1);
  FMMPC_CUDA(cudaMemcpyAsync(T.bmat, B.data(), B.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.dxs, dxs.data(), sizeof(int) * dxs.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(T.err, 0, sizeof(int), H.stream));
  if (W == 24) {
    FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<0, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
    FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<1, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
  } else {
    FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<0, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
    FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
  }
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
  T.enabled = true;
}

// L~ of every volume cell from its M2L list (levels 0-1 cleared); Mv, Lv FP32.
int run_m2l_tc(fmmpc_handle &H, const void *Mv, void *Lv, int nrhs, cudaStream_t s) {
  const TcM2L &T = H.tcm;
  const Geo &g = H.g;
  M2lArgs a{};
  a.img = T.img;
  a.bmat = T.bmat;
  a.tiles = T.tiles;
  a.groups = T.groups;
  a.dxs = T.dxs;
  a.Lv = (cpx<float> *)Lv;
  a.err = T.err;
  a.rows_per_rhs = T.rows_per_rhs;
  a.ncell = g.ncell;
  for (int l = 0; l < 24; ++l) {
    a.lev_row0[l] = T.lev_row0[l];
    a.lev_P[l] = T.lev_P[l];
  }
  for (int q = 0; q < 3; ++q) {
    a.gpart[q] = T.gpart[q];
    a.gpart_sh[q] = T.gpart_sh[q];
  }
  a.p = g.p;
  a.n = g.n;
  a.nsplit = T.nsplit;
  a.nparts = T.nparts;
  a.sbase = T.sbase;
  a.nks = T.kind == 0 ? (T.sbase + 4 * T.nsplit + 7) / 8 : (T.sbase + 4 * T.nsplit + 15) / 16;
  const int64_t lo = level_offset(2), hi = level_offset(g.L + 1);
  const int64_t threads = std::max<int64_t>((int64_t)nrhs * (hi - lo) * 8, (int64_t)nrhs * lo * g.p);
  const cpx<float> *M = (const cpx<float> *)Mv;
  if (T.kind == 0) k_m2l_pack<0><<<nblk(threads), 256, 0, s>>>(a, nrhs, lo, hi, M);
  else k_m2l_pack<1><<<nblk(threads), 256, 0, s>>>(a, nrhs, lo, hi, M);
  FMMPC_LAUNCH_CHECK();
  dim3 grid((unsigned)T.ntiles, (unsigned)T.nparts, (unsigned)nrhs);
  if (T.width == 24) {
    if (T.kind == 0) k_m2l_tc<0, 24><<<grid, M2L_THREADS, T.smem, s>>>(a);
    else k_m2l_tc<1, 24><<<grid, M2L_THREADS, T.smem, s>>>(a);
  } else {
    if (T.kind == 0) k_m2l_tc<0, 32><<<grid, M2L_THREADS, T.smem, s>>>(a);
    else k_m2l_tc<1, 32><<<grid, M2L_THREADS, T.smem, s>>>(a);
  }
  FMMPC_LAUNCH_CHECK();
  return 2;
}

}  // namespace fmmpc
