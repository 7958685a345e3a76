// Lattice near field (P2P, Sec. 5.1 Eq. e:volume_integral restricted to neighbouring leaves)
// on the tensor cores.
//
// On the uniform grid the kernel between a target node of leaf X and a source node of
// leaf X + o depends only on their offset, so for each stencil offset o the near field is
// a matrix product: D[leaf][t] += sum_k W[leaf + o][k] * B_o[t][k], B_o[t][k] = ln|d(t, k, o)|
// (node units, cell-mean value at d = 0), t, k the 64 nodes of an 8x8 leaf.  One CTA takes
// 128 consecutive target leaves of one leaf row (M = 128, N = 64) and sweeps the 37 stencil
// offsets, K = the 64 source nodes of a leaf.
//
// FP32 accuracy from FP16 operands: each operand is split hi + lo (both FP16, rounded to
// nearest; an FP16 word has the 11-bit significand of a TF32 word, so hi + lo carries 22
// bits) and the product is taken as hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32
// rounding).  FP16's narrow exponent range is met by scaling each source leaf's 64 weights
// by a power of two 2^e chosen from the leaf's largest |h^2 r|, so that it lies in
// [2^13, 2^14); the epilogue scales each offset's sums back by the source leaf's 2^-e
// (exact) as it adds them up.  Against TF32 operands the same three products move half the
// bytes and run at twice the rate, and a leaf's 64 source nodes fill one 128-byte row.
//
// The tensor core truncates when it adds into its FP32 accumulator, so a long chain of
// MMAs into one accumulator drifts (~2^-24 of the partial sum per MMA).  Each offset's group
// therefore starts a fresh accumulator -- the two small correction products first, the
// hi*hi products last -- and four epilogue warps drain it into per-thread FP32 sums while
// the next groups run in the other TMEM buffers (four in flight).  The stencil rows are
// split between two CTAs (the second writes a scratch image that the L2P pass adds), and
// two CTAs share an SM, so one's copies and barrier round trips overlap the other's MMAs.
//
// Data: per padded leaf row, each leaf's 64 scaled weights are one 128-byte row in the
// 128-byte swizzle (16-byte chunk c of leaf X at position c ^ (X % 8)), leaves contiguous,
// so the 134 leaves a tile needs are one 1-D bulk copy straight into the MMA operand layout,
// and a shift by ox leaves is a 128-byte shift of the descriptor start.  The B_o pairs
// (hi, lo) are precomputed in the same layout (16 KB per offset).  Warp 0 streams strips
// (two slots) and B groups (two slots); warp 1 issues the MMAs; warps 2-5 drain TMEM.
#include <cmath>
#include <cstring>

#include <cuda_fp16.h>

#include "handle.cuh"
#include "tc.cuh"

namespace fmmpc {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

constexpr int TC_TILE = 128;       // target leaves per CTA
constexpr int TC_BGRP = 16384;     // one offset's B: hi + lo, 64 x 64 FP16 each
constexpr int TC_NB = 2;           // B stages per CTA (two CTAs per SM)
constexpr int TC_NACC = 4;         // TMEM accumulators (64 columns each) in flight
constexpr int TC_THREADS = 192;    // producer, MMA issuer, four epilogue warps
constexpr int TC_MAXROWS = 33;
constexpr int TC_TOP = 13;         // the largest scaled weight lies in [2^TC_TOP, 2^(TC_TOP+1))

// instruction descriptor of tcgen05.mma kind::f16 with FP16 A and B, FP32 accumulation,
// K-major operands: bits 4-5 D format (1 = F32), 7-9 / 10-12 A / B format (0 = F16),
// 17-22 N >> 3, 24-28 M >> 4
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t M, uint32_t N) { return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24); }

struct TcArgs {
  const uint16_t *ahi, *alo;  // [nrhs][NLY][NLX][64] FP16, swizzled per leaf
  const uint16_t *bmat;       // [nofs][hi, lo][64][64] FP16, swizzled per row t
  const float *lsc;           // [nrhs][NLY][NLX] 2^-e of each (padded) source leaf
  float *out1, *out2;  // near-field sums (unscaled), first and second part of the stencil rows
  int *err;
  int n, R, NLX, NLY, NS, nrows, nofs, npass, usplit;
  int row_oy[TC_MAXROWS], row_q0[TC_MAXROWS], row_q1[TC_MAXROWS], row_ox0[TC_MAXROWS];
};

// h^2 as two FP32 words for the weight product
inline float h2_hi(double h) { return (float)(h * h); }
inline float h2_lo(double h) { return (float)(h * h - (double)(float)(h * h)); }

// w = fl32(h^2 r) from a two-word FP32 product (h^2 and r each as hi + lo, the product of
// the high words split exactly by an FMA): the FP32 weight of the CUDA-core engine's image
__device__ __forceinline__ float weight_of(double r, float h2h, float h2l) {
  const float2 x2 = f64_to_f32x2(r);
  const float xh = x2.x, xl = x2.y;
  const float p = __fmul_rn(xh, h2h);
  const float t = fmaf(xh, h2l, fmaf(xl, h2h, fmaf(xh, h2h, -p)));
  return p + t;
}

// Weight strips: node (i, j) -> leaf (X, Y) = (i/8 + R, j/8 + R), k = (j%8) 8 + i%8.  Thread
// per (rhs, leaf, node row jr = j%8 of the leaf), jr fastest, so the eight lanes of a leaf
// find its largest |w| by three shuffles.  Each writes its row's FP16 hi and lo words (the
// weights times the leaf's 2^e) as 16-byte chunk jr of the leaf's swizzled 128-byte rows,
// so a leaf's eight lanes write whole rows, and the same 8 weights unscaled into the FP32
// zero-padded weight image the other stages read (w, npad, pad).  lsc gets the leaf's 2^-e.
// 2^e puts the leaf's largest weight in [2^TC_TOP, 2^(TC_TOP+1)); e is capped at 126 so that
// 2^e and 2^-e stay FP32 numbers (a leaf whose largest weight is below 2^-113 keeps fewer
// than 22 bits in the split; its near field is within a few FP32 ulps of underflow anyway).
__global__ void k_tc_strips(int n, int lgNL, int R, int NLX, int NLY, float h2h, float h2l, int nrhs,
                            const double *__restrict__ r, uint16_t *__restrict__ ahi, uint16_t *__restrict__ alo,
                            float *__restrict__ lsc, float *__restrict__ wimg, int npad, int pad) {
  const int NL = 1 << lgNL;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < ((int64_t)nrhs << (2 * lgNL + 3));  // every lane takes part in the shuffles
  const int jr = (int)(t & 7);
  const int Xl = (int)((t >> 3) & (NL - 1));
  const int Yl = (int)((t >> (3 + lgNL)) & (NL - 1));
  const int64_t rhs = t >> (3 + 2 * lgNL);
  const int X = Xl + R, Y = Yl + R;
  const int64_t leaf = (rhs * NLY + Y) * NLX + X, rowoff = leaf * 64;
  const int j = 8 * Yl + jr, i0 = 8 * Xl;
  const double *src = r + rhs * (int64_t)n * n + (int64_t)j * n + i0;
  float w[8];
  float m = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    w[q] = in ? weight_of(src[q], h2h, h2l) : 0.0f;
    m = fmaxf(m, fabsf(w[q]));
  }
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
  // floor(log2 m) from the FP32 fields (a subnormal m counts as 2^-127: e is capped anyway)
  const int e = m > 0.0f ? min(TC_TOP - ((int)((__float_as_uint(m) >> 23) & 0xffu) - 127), 126) : 0;
  const float sc = ldexpf(1.0f, e);
  if (!in) return;
  if (jr == 0) lsc[leaf] = ldexpf(1.0f, -e);
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    const float a = w[q] * sc, b = w[q + 1] * sc;  // exact: scaling by a power of two
    const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
    const __half al = __float2half_rn(a - __half2float(ah)), bl = __float2half_rn(b - __half2float(bh));
    hw[q / 2] = (uint32_t)__half_as_ushort(ah) | ((uint32_t)__half_as_ushort(bh) << 16);
    lw[q / 2] = (uint32_t)__half_as_ushort(al) | ((uint32_t)__half_as_ushort(bl) << 16);
  }
  const int pos = jr ^ (X & 7);
  reinterpret_cast<uint4 *>(ahi + rowoff)[pos] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  reinterpret_cast<uint4 *>(alo + rowoff)[pos] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  float *wr = wimg + rhs * (int64_t)npad * npad + (int64_t)(j + pad) * npad + i0 + pad;
  reinterpret_cast<float4 *>(wr)[0] = make_float4(w[0], w[1], w[2], w[3]);
  reinterpret_cast<float4 *>(wr)[1] = make_float4(w[4], w[5], w[6], w[7]);
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_p2p_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full_s[2], empty_s[2], full_b[TC_NB], empty_b[TC_NB], acc_full[TC_NACC], acc_empty[TC_NACC], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, used_s, used_b;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int SH = (a.NS * 128 + 1023) & ~1023;  // bytes of one strip (hi or lo)
  // the swizzle is taken from absolute address bits: operands start on 1024-byte boundaries
  unsigned char *strips = smem + ((1024u - (tc::smem_addr(smem) & 1023u)) & 1023u);  // [2][hi, lo][SH]
  unsigned char *bm = strips + 4 * SH;                                                 // [TC_NB][TC_BGRP]
  const int lx0 = blockIdx.x * TC_TILE, ly = blockIdx.y, rhs = blockIdx.z >> 1, half = blockIdx.z & 1;
  // this CTA's stencil rows [u0, u1); the other part goes to a.out2
  const int u0 = half ? a.usplit : 0, u1 = half ? a.nrows : a.usplit;
  int ngroups = 0;
  for (int u = u0; u < u1; ++u) ngroups += a.row_q1[u] - a.row_q0[u];
  // Every CTA sweeps the same stencil rows; started in step they would all read the same B
  // group from the same few L2 slices at the same time.  The CTAs of leaf row ly therefore
  // take their rows from row (ly mod nr) on, wrapping around: the lu-th row of the sweep is
  // urow(lu).  The order of the sums is fixed per leaf row and the same for every
  // right-hand side.
  const int nr = u1 - u0, rot = nr > 0 ? ly % nr : 0;
  auto urow = [&](int lu) { return u0 + (lu + rot < nr ? lu + rot : lu + rot - nr); };
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&full_s[b], 1);
      tc::mbar_init(&empty_s[b], 1);
    }
    for (int b = 0; b < TC_NACC; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 4);
    }
    for (int b = 0; b < TC_NB; ++b) {
      tc::mbar_init(&full_b[b], 1);
      tc::mbar_init(&empty_b[b], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_init_fence();
    abort_flag = 0;
    used_s = 0;
    used_b = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, 64 * TC_NACC);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const int64_t rhs_off = (int64_t)rhs * a.NLY * a.NLX * 64;
  int issued_s = 0, issued_b = 0;
  if (warp == 0) {
    if (lane == 0) {
      // producer: per stencil row the weight strip, then that row's B groups
      int g = 0;
      bool ok = true;
      for (int lu = 0; lu < nr && ok && !abort_flag; ++lu) {
        const int u = urow(lu), slot = lu & 1;
        if (lu >= 2 && !tc::mbar_wait(&empty_s[slot], ((lu >> 1) - 1) & 1, &abort_flag)) { ok = false; break; }
        tc::mbar_expect_tx(&full_s[slot], 2 * a.NS * 128);
        const int64_t Y = ly + a.R + a.row_oy[u];
        const int64_t off = rhs_off + (Y * a.NLX + lx0) * 64;
        tc::bulk_g2s(strips + (slot * 2) * SH, a.ahi + off, a.NS * 128, &full_s[slot]);
        tc::bulk_g2s(strips + (slot * 2 + 1) * SH, a.alo + off, a.NS * 128, &full_s[slot]);
        issued_s = lu + 1;
        for (int q = a.row_q0[u]; q < a.row_q1[u]; ++q) {
          const int bi = g % TC_NB;
          if (g >= TC_NB && !tc::mbar_wait(&empty_b[bi], ((g / TC_NB) - 1) & 1, &abort_flag)) { ok = false; break; }
          tc::mbar_expect_tx(&full_b[bi], TC_BGRP);
          tc::bulk_g2s(bm + bi * TC_BGRP, a.bmat + (int64_t)q * (TC_BGRP / 2), TC_BGRP, &full_b[bi]);
          issued_b = ++g;
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: one fresh accumulator per offset group, four buffers in turn
      const uint32_t idesc = idesc_f16(128, 64);
      // descriptor low words (+8 per 128-byte row, +2 per K step of 16 FP16 values)
      const uint32_t slo0 = tc::desc_lo(tc::smem_addr(strips)), blo0 = tc::desc_lo(tc::smem_addr(bm));
      int g = 0;
      bool ok = true;
      for (int lu = 0; lu < nr && ok; ++lu) {
        const int u = urow(lu), slot = lu & 1;
        if (!tc::mbar_wait(&full_s[slot], (lu >> 1) & 1, &abort_flag)) { ok = false; break; }
        used_s = lu + 1;
        tc::fence_after();
        // strips (hi, lo) of this slot, shifted to the row's first offset
        const uint32_t shlo = slo0 + (uint32_t)((slot * 2) * (SH >> 4) + (a.R + a.row_ox0[u]) * 8);
        const uint32_t sllo = shlo + (uint32_t)(SH >> 4);
        const int q0 = a.row_q0[u], q1 = a.row_q1[u];
        for (int q = q0; q < q1; ++q) {
          const int bi = g % TC_NB, ab = g % TC_NACC;
          if (!tc::mbar_wait(&full_b[bi], (g / TC_NB) & 1, &abort_flag)) { ok = false; break; }
          used_b = g + 1;
          if (g >= TC_NACC && !tc::mbar_wait(&acc_empty[ab], ((g / TC_NACC) - 1) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t bhl = blo0 + (uint32_t)(bi * (TC_BGRP >> 4)), bll = bhl + (uint32_t)(TC_BGRP / 2 >> 4);
          const uint32_t d = tmem + 64 * ab;
          const uint32_t ahl = shlo + 8u * (uint32_t)(q - q0), all = sllo + 8u * (uint32_t)(q - q0);
          if (a.npass == 3) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              tc::mma_f16(d, tc::desc_of(ahl + 2 * s), tc::desc_of(bll + 2 * s), idesc, s > 0 ? 1u : 0u);
              tc::mma_f16(d, tc::desc_of(all + 2 * s), tc::desc_of(bhl + 2 * s), idesc, 1u);
            }
          }
          const uint32_t acc0 = a.npass == 3 ? 1u : 0u;
#pragma unroll
          for (int s = 0; s < 4; ++s)
            tc::mma_f16(d, tc::desc_of(ahl + 2 * s), tc::desc_of(bhl + 2 * s), idesc, s > 0 ? 1u : acc0);
          tc::commit(&acc_full[ab]);  // the epilogue also releases the B and strip slots
          ++g;
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
      tc::commit(&done);  // completes when every MMA issued above has finished
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one target leaf per thread
    const int qd = warp & 3;
    float sum[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) sum[i] = 0.0f;
    bool ok = true;
    int lu = 0, u = urow(0), uend = a.row_q1[u] - a.row_q0[u];  // groups of the current row end at uend
    // 2^-e of this thread's source leaf for offset (ox, oy): row of the padded leaf grid
    const int Xp = lx0 + 32 * qd + lane + a.R;
    const float *lrow = a.lsc + ((int64_t)rhs * a.NLY + ly + a.R) * a.NLX + Xp;
    for (int g = 0; g < ngroups; ++g) {
      const int ab = g % TC_NACC;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc_full[ab], (g / TC_NACC) & 1, &abort_flag))) {
        ok = false;  // warp-uniform: the TMEM loads below are warp-collective
        break;
      }
      if (warp == 2 && lane == 0) {
        // the group's MMAs have completed: its B slot, and at a row's end the strip slot, are free
        tc::mbar_arrive(&empty_b[g % TC_NB]);
        if (g + 1 == uend) tc::mbar_arrive(&empty_s[lu & 1]);
      }
      const int nu = a.row_q1[u] - a.row_q0[u];
      const int ox = a.row_ox0[u] + (g - (uend - nu)), oy = a.row_oy[u];
      const float us = __ldg(lrow + (int64_t)oy * a.NLX + ox);
      if (g + 1 == uend && ++lu < nr) {
        u = urow(lu);
        uend += a.row_q1[u] - a.row_q0[u];
      }
      tc::fence_after();
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * ab + 32 * hf, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) sum[32 * hf + i] = fmaf(v[i], us, sum[32 * hf + i]);  // v 2^-e exact
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[ab]);
    }
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicOr(a.err, 2);
    }
    if (ok && !abort_flag) {
      const int X = lx0 + 32 * qd + lane;
      // the part's sum as accumulated: the -1/(2 pi) and the sum of the two parts are applied
      // once, in FP64, where the near field meets the far field
      float *o = (half ? a.out2 : a.out1) + (int64_t)rhs * a.n * a.n + (int64_t)(ly * 8) * a.n + X * 8;
#pragma unroll
      for (int tr = 0; tr < 8; ++tr) {
        float4 *orow = reinterpret_cast<float4 *>(o + (int64_t)tr * a.n);
        orow[0] = make_float4(sum[8 * tr], sum[8 * tr + 1], sum[8 * tr + 2], sum[8 * tr + 3]);
        orow[1] = make_float4(sum[8 * tr + 4], sum[8 * tr + 5], sum[8 * tr + 6], sum[8 * tr + 7]);
      }
    }
  }
  __syncwarp();
  const bool finished = tc::mbar_wait(&done, 0, nullptr);
  if (!finished && lane == 0) atomicOr(a.err, 4);
  tc::fence_before();
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0) {
    // drain bulk copies that were issued but never consumed (bounded waits)
    for (int u = used_s; u < issued_s; ++u) tc::mbar_wait(&full_s[u & 1], (u >> 1) & 1, nullptr);
    for (int u = used_b; u < issued_b; ++u) tc::mbar_wait(&full_b[u % TC_NB], (u / TC_NB) & 1, nullptr);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 64 * TC_NACC);
  }
}

__global__ void k_near_combine(int64_t total, const float *__restrict__ a, const float *__restrict__ b,
                               double *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) out[t] = ((double)a[t] + (double)b[t]) * NEG_INV_2PI;
}

// FP16 word of v, rounded to nearest even (host; v within FP16's normal range)
uint16_t f16_round_host(double v) {
  const __half h = __float2half_rn((float)v);
  return __half_as_ushort(h);
}

double f16_value_host(uint16_t b) { return (double)__half2float(__ushort_as_half(b)); }

}  // namespace

bool tc_p2p_eligible(const fmmpc_handle &H) {
  const Geo &g = H.g;
  return g.m == 8 && H.prec != FMMPC_PREC_FP64 && (1 << g.L) >= TC_TILE && 2 * g.R + 1 <= TC_MAXROWS;
}

void init_tc_p2p(fmmpc_handle &H) {
  H.tcp.enabled = tc_p2p_eligible(H);
  if (!H.tcp.enabled) return;
  const Geo &g = H.g;
  const Stencil &st = H.st;
  const int NL = (1 << g.L) + 2 * g.R;
  H.tcp.NLX = NL;
  H.tcp.NLY = NL;
  H.tcp.NS = TC_TILE + 2 * g.R;
  H.tcp.npass = 3;  // the near field stays FP32-accurate in every single-precision form
  const size_t strip_words = (size_t)H.nrhs_max * NL * NL * 64;
  H.tcp.ahi = H.pool.get<uint16_t>(strip_words);
  H.tcp.alo = H.pool.get<uint16_t>(strip_words);
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.ahi, 0, sizeof(uint16_t) * strip_words, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.alo, 0, sizeof(uint16_t) * strip_words, H.stream));
  // B pairs for every stencil offset, rows in the order (oy, ox); without and with ln h
  std::vector<int> oys, q0s, q1s, ox0s;
  int nofs = 0;
  for (int oy = -st.R; oy <= st.R; ++oy) {
    const int a0 = st.ox0[oy + st.R], a1 = st.ox1[oy + st.R];
    if (a0 > a1) continue;
    oys.push_back(oy);
    q0s.push_back(nofs);
    ox0s.push_back(a0);
    nofs += a1 - a0 + 1;
    q1s.push_back(nofs);
  }
  H.tcp.nrows = (int)oys.size();
  for (int r = 0; r < H.tcp.nrows; ++r) {
    H.tcp.row_oy[r] = oys[r];
    H.tcp.row_q0[r] = q0s[r];
    H.tcp.row_q1[r] = q1s[r];
    H.tcp.row_ox0[r] = ox0s[r];
  }
  const double cself = -0.5 * std::log(2.0) - 1.5 + 0.25 * PI;
  for (int variant = 0; variant < 2; ++variant) {
    // offset q: [hi: 64 rows t][64 k] swizzled, then [lo: same]
    std::vector<uint16_t> B((size_t)nofs * (TC_BGRP / 2), 0);
    for (int r = 0; r < H.tcp.nrows; ++r)
      for (int q = q0s[r]; q < q1s[r]; ++q) {
        const int ox = ox0s[r] + (q - q0s[r]), oy = oys[r];
        uint16_t *Bg = B.data() + (size_t)q * (TC_BGRP / 2);
        for (int t = 0; t < 64; ++t)
          for (int k = 0; k < 64; ++k) {
            const int dx = (t % 8) - (k % 8) - 8 * ox, dy = (t / 8) - (k / 8) - 8 * oy;
            double v = (dx == 0 && dy == 0) ? cself : 0.5 * std::log((double)dx * dx + (double)dy * dy);
            if (variant) v += g.lnh;
            const uint16_t hi = f16_round_host(v);
            const size_t e = (size_t)t * 64 + (((k / 8) ^ (t & 7)) * 8) + (k % 8);
            Bg[e] = hi;
            Bg[TC_BGRP / 4 + e] = f16_round_host(v - f16_value_host(hi));
          }
      }
    uint16_t *dB = H.pool.get<uint16_t>(B.size());
    FMMPC_CUDA(cudaMemcpyAsync(dB, B.data(), sizeof(uint16_t) * B.size(), cudaMemcpyHostToDevice, H.stream));
    FMMPC_CUDA(cudaStreamSynchronize(H.stream));
    (variant ? H.tcp.bmat_lnh : H.tcp.bmat) = dB;
  }
  H.tcp.nofs = nofs;
  {  // split the stencil rows into two parts of about equal offset counts
    int acc = 0, best = 1, bestd = 1 << 30;
    for (int u = 0; u < H.tcp.nrows; ++u) {
      acc += q1s[u] - q0s[u];
      const int d = std::abs(2 * acc - nofs);
      if (u + 1 < H.tcp.nrows && d < bestd) { bestd = d; best = u + 1; }
    }
    H.tcp.usplit = best;
  }
  H.tcp.near1 = H.pool.get<float>((size_t)H.nrhs_max * g.n * g.n);
  H.tcp.near2 = H.pool.get<float>((size_t)H.nrhs_max * g.n * g.n);
  H.tcp.lsc = H.pool.get<float>((size_t)H.nrhs_max * NL * NL);
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.lsc, 0, sizeof(float) * H.nrhs_max * NL * NL, H.stream));  // padding leaves
  H.tcp.err = H.pool.get<int>(1);
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.err, 0, sizeof(int), H.stream));
  const int smem = 4 * ((H.tcp.NS * 128 + 1023) & ~1023) + TC_NB * TC_BGRP + 1024;  // + alignment slack
  FMMPC_CUDA(cudaFuncSetAttribute(k_p2p_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  H.tcp.smem = smem;
}

// FP16 hi/lo weight strips of the right-hand side r (FP64) with their per-leaf scales, for
// run_p2p_tc, and the FP32 weight image, in one pass.
int prep_p2p_tc(fmmpc_handle &H, const double *r, int nrhs, cudaStream_t s, float *wimg) {
  const Geo &g = H.g;
  const int lgNL = g.L;  // n / 8 = 2^L leaves per side (8 x 8 leaves)
  const int64_t threads = ((int64_t)nrhs << (2 * lgNL)) * 8;
  k_tc_strips<<<nblk(threads), 256, 0, s>>>(g.n, lgNL, g.R, H.tcp.NLX, H.tcp.NLY, h2_hi(g.h), h2_lo(g.h), nrhs, r,
                                            H.tcp.ahi, H.tcp.alo, H.tcp.lsc, wimg, g.npad, g.pad);
  FMMPC_LAUNCH_CHECK();
  return 1;
}

// out[...] = -near / (2 pi) on the tensor cores, from the strips prep_p2p_tc wrote.
int run_p2p_tc(fmmpc_handle &H, bool with_lnh, double *out, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  TcArgs a{};
  a.ahi = H.tcp.ahi;
  a.alo = H.tcp.alo;
  a.bmat = with_lnh ? H.tcp.bmat_lnh : H.tcp.bmat;
  a.lsc = H.tcp.lsc;
  a.out1 = H.tcp.near1;
  (void)out;
  a.err = H.tcp.err;
  a.n = g.n;
  a.R = g.R;
  a.NLX = H.tcp.NLX;
  a.NLY = H.tcp.NLY;
  a.NS = H.tcp.NS;
  a.nrows = H.tcp.nrows;
  a.nofs = H.tcp.nofs;
  a.usplit = H.tcp.usplit;
  a.out2 = H.tcp.near2;
  a.npass = H.tcp.npass;
  for (int i = 0; i < a.nrows; ++i) {
    a.row_oy[i] = H.tcp.row_oy[i];
    a.row_q0[i] = H.tcp.row_q0[i];
    a.row_q1[i] = H.tcp.row_q1[i];
    a.row_ox0[i] = H.tcp.row_ox0[i];
  }
  dim3 grid((1 << g.L) / TC_TILE, 1 << g.L, 2 * nrhs);
  k_p2p_tc<<<grid, TC_THREADS, H.tcp.smem, s>>>(a);
  FMMPC_LAUNCH_CHECK();
  return 1;
}

// out = the two parts of the near field (PART_NEAR, where no L2P pass follows).
int add_near2(fmmpc_handle &H, double *out, int nrhs, cudaStream_t s) {
  const int64_t total = (int64_t)H.g.n * H.g.n * nrhs;
  k_near_combine<<<nblk(total), 256, 0, s>>>(total, H.tcp.near1, H.tcp.near2, out);
  FMMPC_LAUNCH_CHECK();
  return 1;
}

}  // namespace fmmpc
