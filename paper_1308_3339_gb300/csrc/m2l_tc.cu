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
// multipole image with 140 fixed matrices.  The image of each level is split into its four
// parity sub-images, each zero-padded by 4 cells and flattened with row pitch P = S + 8
// (S = 2^(l-1) cells), so that for a target class and an offset the sources of 128
// consecutive flattened targets are 128 consecutive rows of one sub-image, shifted by
// dy P + dx.  One CTA takes such a tile of targets (M = 128) and sweeps its class's offsets,
// D[t][u] += sum_v X[t + shift][v] B_o[u][v] with K = 2p real inputs and N = 32 outputs: 2p
// real parts of L~ plus the two sums of M~_0 that carry the ln rho term.  Padding targets are
// computed and dropped.  The low-order terms dominate the translated
// field and meets the large log o + ln rho, so their products are split hi + lo in the
// spare K columns (K = 32 for TF32: M~_0..2 at p = 10; K = 48 for BF16: M~_0..6): rounded input x rounded
// matrix, input residual x rounded matrix, rounded input x matrix residual.
//
// Operands use the 128-byte swizzle (one 128-byte row per cell), so a shifted window is a
// descriptor offset.  Offsets are grouped by (source parity, dy); one 144-row window of the
// source sub-image serves every dx of a group.  Warp 0 streams window + B groups through
// two stages (two CTAs share an SM, so their copy and MMA round trips overlap), warp 1
// issues the MMAs, one fresh TMEM accumulator per group (four in
// flight), and warps 2-5 drain each into Kahan-compensated FP32 sums: one long chain of
// MMAs would drift with the tensor core's truncating adds (~2^-24 of the partial per MMA).
#include <algorithm>
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
constexpr int M2L_BBYTES = 32 * 128;            // one offset's B operand: 32 outputs x 128 B
constexpr int M2L_NSTG = 2;                     // stages per CTA (two CTAs per SM)
constexpr int M2L_NACC = 4;                     // TMEM accumulators (32 columns each) in flight
constexpr int M2L_THREADS = 192;
constexpr int M2L_TAIL = 256;                   // zero rows after each sub-image (window overrun)
constexpr int M2L_MAXGRP = 128, M2L_MAXOFS = 225;  // per class: (source parity, dy) groups, offsets

struct M2lArgs {
  const unsigned char *img;     // [nrhs][rows_per_rhs][128 B]
  const unsigned char *bmat;    // [class][offset][32][128 B]
  const int4 *tiles;            // (level, class, f0, -)
  const int4 *groups;           // [class][group]: (source parity, dy, first offset, count)
  const int *dxs;               // [class][offset]: dx of the offset
  cpx<float> *Lv;               // [nrhs][ncell][p]
  int *err;
  int64_t rows_per_rhs, ncell;
  int64_t lev_row0[24];         // first image row of level l (parity 0)
  int lev_P[24];
  int ngroups[4], goff[4], ooff[4], nofs[4];
  int p, n, stage_bytes, nks, nsplit;
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
// for j < nsplit, v = 2p + 4j + {0, 1}: the rounding residual of M~_j (meets B's rounded
// column j), v = 2p + 4j + {2, 3}: the rounded M~_j again (meets the residual of column j).
template <int KIND>
__device__ __forceinline__ float m2l_input(const cpx<float> *M, int v, int p, int nsplit) {
  if (v < 2 * p) {
    const float x = (v & 1) ? M[v >> 1].im : M[v >> 1].re;
    return m2l_round<KIND>(x);
  }
  const int w = v - 2 * p, j = w >> 2, e = w & 3;
  if (j >= nsplit) return 0.f;
  const float x = (e & 1) ? M[j].im : M[j].re;
  const float hi = m2l_round<KIND>(x);
  return e < 2 ? m2l_round<KIND>(x - hi) : hi;
}

// Multipole image rows: thread per (rhs, cell at level >= 2, 16-byte chunk).  Also clears
// the local expansions of levels 0 and 1, which have no M2L sources.
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
  uint32_t w[4];
  if (KIND == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = __float_as_uint(m2l_input<KIND>(M, 4 * chunk + e, a.p, a.nsplit));
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 b0 = __float2bfloat16_rn(m2l_input<KIND>(M, 8 * chunk + 2 * e, a.p, a.nsplit));
      const __nv_bfloat16 b1 = __float2bfloat16_rn(m2l_input<KIND>(M, 8 * chunk + 2 * e + 1, a.p, a.nsplit));
      w[e] = (uint32_t)*reinterpret_cast<const uint16_t *>(&b0) | ((uint32_t)*reinterpret_cast<const uint16_t *>(&b1) << 16);
    }
  }
  uint4 *dst = reinterpret_cast<uint4 *>(const_cast<unsigned char *>(a.img) + row * 128) + (chunk ^ (int)(f & 7));
  *dst = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int KIND>
__global__ void __launch_bounds__(M2L_THREADS, 2) k_m2l_tc(M2lArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t full[M2L_NSTG], empty[M2L_NSTG], acc_full[M2L_NACC], acc_empty[M2L_NACC], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, used;
  __shared__ int4 sgrp[M2L_MAXGRP];  // the class's groups and offsets, off the issue path
  __shared__ int sdx[M2L_MAXOFS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int4 tile = a.tiles[blockIdx.x];
  const int l = tile.x, c = tile.y, f0 = tile.z, rhs = blockIdx.y;
  const int P = a.lev_P[l];
  const int ng = a.ngroups[c];
  for (int i = tid; i < ng; i += blockDim.x) sgrp[i] = a.groups[a.goff[c] + i];
  for (int i = tid; i < a.nofs[c]; i += blockDim.x) sdx[i] = a.dxs[a.ooff[c] + i];
  const int4 *grp = sgrp;
  if (tid == 0) {
    for (int s = 0; s < M2L_NSTG; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < M2L_NACC; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 4);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_init_fence();
    abort_flag = 0;
    used = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, 32 * M2L_NACC);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      // producer: per group, the source window and the group's B operands into one stage
      bool ok = true;
      for (int gi = 0; gi < ng && !abort_flag; ++gi) {
        const int s = gi % M2L_NSTG;
        if (gi >= M2L_NSTG && !tc::mbar_wait(&empty[s], ((gi / M2L_NSTG) - 1) & 1, &abort_flag)) { ok = false; break; }
        const int4 g = grp[gi];  // (source parity, dy, first, count)
        const int ws = floor8(f0 + g.y * P - 4);
        const unsigned char *src = a.img + ((int64_t)rhs * a.rows_per_rhs + a.lev_row0[l] +
                                            (int64_t)g.x * ((int64_t)P * P + M2L_TAIL) + ws) * 128;
        unsigned char *st = smem + s * a.stage_bytes;
        tc::mbar_expect_tx(&full[s], M2L_WBYTES + g.w * M2L_BBYTES);
        tc::bulk_g2s(st, src, M2L_WBYTES, &full[s]);
        tc::bulk_g2s(st + M2L_WBYTES, a.bmat + ((int64_t)a.ooff[c] + g.z) * M2L_BBYTES, g.w * M2L_BBYTES, &full[s]);
        issued = gi + 1;
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: one fresh accumulator per group; one commit per group (the epilogue,
      // which waits for the same completion, releases the stage)
      const uint32_t idesc = KIND == 0 ? tc::idesc_tf32(128, 32)
                                       : ((1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24));
      const int nks = a.nks;  // K steps of 32 bytes (8 TF32 or 16 BF16 inputs each)
      bool ok = true;
      for (int gi = 0; gi < ng; ++gi) {
        const int s = gi % M2L_NSTG, ab = gi % M2L_NACC;
        if (!tc::mbar_wait(&full[s], (gi / M2L_NSTG) & 1, &abort_flag)) { ok = false; break; }
        used = gi + 1;
        if (gi >= M2L_NACC && !tc::mbar_wait(&acc_empty[ab], ((gi / M2L_NACC) - 1) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const int4 g = grp[gi];
        const int ws = floor8(f0 + g.y * P - 4);
        const uint32_t st = tc::smem_addr(smem + s * a.stage_bytes);
        const uint32_t d = tmem + 32 * ab;
        uint32_t acc = 0;
        for (int k = 0; k < g.w; ++k) {
          const int dx = sdx[g.z + k];
          const uint32_t arow = st + (uint32_t)((f0 + g.y * P + dx - ws) * 128);
          const uint32_t brow = st + M2L_WBYTES + k * M2L_BBYTES;
          for (int ks = 0; ks < nks; ++ks) {
            const uint64_t ad = tc::desc_sw128(arow + 32 * ks), bd = tc::desc_sw128(brow + 32 * ks);
            if (KIND == 0) {
              tc::mma_tf32(d, ad, bd, idesc, acc);
            } else {
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            acc = 1;
          }
        }
        tc::commit(&acc_full[ab]);
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(a.err, 1);
      }
      tc::commit(&done);
    }
  } else {
    // epilogue: drain each group's accumulator into FP32 sums (Kahan), one target per thread
    const int qd = warp & 3;
    float sum[32], cmp[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) sum[i] = cmp[i] = 0.0f;
    bool ok = true;
    for (int gi = 0; gi < ng; ++gi) {
      const int ab = gi % M2L_NACC;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&acc_full[ab], (gi / M2L_NACC) & 1, &abort_flag))) {
        ok = false;
        break;
      }
      tc::fence_after();
      if (warp == 2 && lane == 0) tc::mbar_arrive(&empty[gi % M2L_NSTG]);  // the group's MMAs are done
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 32 * ab, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float y = v[i] - cmp[i];
        const float t = sum[i] + y;
        cmp[i] = (t - sum[i]) - y;
        sum[i] = t;
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
      const int x = 2 * i + (c & 1), y = 2 * j + (c >> 1);
      const int64_t gidx = level_offset(l) + morton_encode((uint32_t)x, (uint32_t)y);
      cpx<float> *L = a.Lv + ((int64_t)rhs * a.ncell + gidx) * a.p;
      const float lnrho = logf((float)(a.n >> l));
      float tot[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) tot[u] = sum[u] - cmp[u];
      float m0r = 0.f, m0i = 0.f;  // the sums of M~_0 in outputs 2p, 2p + 1 (p <= 15)
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        if (u == 2 * a.p) m0r = tot[u];
        if (u == 2 * a.p + 1) m0i = tot[u];
      }
      L[0] = mk<float>(tot[0] + lnrho * m0r, tot[1] + lnrho * m0i);
#pragma unroll
      for (int nn = 1; nn < 16; ++nn)
        if (nn < a.p) L[nn] = mk<float>(tot[2 * nn], tot[2 * nn + 1]);
    }
  }
  __syncwarp();
  const bool finished = __all_sync(0xffffffffu, tc::mbar_wait(&done, 0, nullptr));  // warp-uniform
  if (!finished && lane == 0) atomicOr(a.err, 4);
  tc::fence_before();
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0)
    for (int u = used; u < issued; ++u) tc::mbar_wait(&full[u % M2L_NSTG], (u / M2L_NSTG) & 1, nullptr);
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 32 * M2L_NACC);
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
  // N = 32 outputs hold 2p + 2; K (32 TF32 or BF16 inputs per 128-byte row) holds 2p
  return (H.prec == FMMPC_PREC_MIXED_BF16 || H.prec == FMMPC_PREC_MIXED_TF32) && H.g.L >= 2 && 2 * H.g.p + 2 <= 32;
}

void init_tc_m2l(fmmpc_handle &H, DevPool &tmp) {
  TcM2L &T = H.tcm;
  T.enabled = false;
  if (!tc_m2l_eligible(H)) return;
  const Geo &g = H.g;
  const int L = g.L, p = g.p;
  T.kind = (H.prec == FMMPC_PREC_MIXED_TF32) ? 0 : 1;
  // hi/lo splits of the leading multipoles in the spare K columns (24 for TF32, 32 for BF16)
  // K capacity: TF32 32 inputs (4 steps of 8, one 128-byte row); BF16 48 (3 steps of 16)
  const int kcap = T.kind == 0 ? 32 : 48;
  T.nsplit = std::max(0, std::min(p, (kcap - 2 * p) / 4));
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
  // per class: offsets sorted by (source parity, dy, dx), grouped by (source parity, dy)
  std::vector<int4> groups;
  std::vector<int> dxs;
  std::vector<std::pair<int, int>> ofs_all;  // (ox, oy) in class order
  int maxcnt = 1;
  for (int c = 0; c < 4; ++c) {
    const int cx = c & 1, cy = c >> 1;
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> bykey;  // (sp, dy) -> (dx, idx)
    for (int oy = -7; oy <= 7; ++oy)
      for (int ox = -7; ox <= 7; ++ox) {
        if (!tab[c * 225 + (oy + 7) * 15 + ox + 7]) continue;
        const int spx = (cx - ox) & 1, spy = (cy - oy) & 1;
        const int dx = (cx - ox - spx) / 2, dy = (cy - oy - spy) / 2;
        bykey[{spx + 2 * spy, dy}].push_back({dx, (oy + 7) * 15 + ox + 7});
      }
    T.goff[c] = (int)groups.size();
    T.ooff[c] = (int)dxs.size();
    int first = 0;
    for (auto &kv : bykey) {
      auto v = kv.second;
      std::sort(v.begin(), v.end());
      groups.push_back(make_int4(kv.first.first, kv.first.second, first, (int)v.size()));
      for (auto &e : v) {
        dxs.push_back(e.first);
        ofs_all.push_back({e.second % 15 - 7, e.second / 15 - 7});
      }
      first += (int)v.size();
      maxcnt = std::max(maxcnt, (int)v.size());
    }
    T.ngroups[c] = (int)groups.size() - T.goff[c];
  }
  T.nofs_total = (int)dxs.size();
  for (int c = 0; c < 4; ++c)
    if (T.ngroups[c] > M2L_MAXGRP) throw Error(FMMPC_ERR_UNSUPPORTED, "tensor-core M2L: too many offset groups");
  // B operands: rows u (2p outputs, then sum Re M0, sum Im M0), columns v (2p inputs)
  std::vector<unsigned char> B((size_t)T.nofs_total * M2L_BBYTES, 0);
  std::vector<double> fact(2 * p + 2, 1.0);
  for (int i = 1; i < (int)fact.size(); ++i) fact[i] = fact[i - 1] * i;
  for (int q = 0; q < T.nofs_total; ++q) {
    const std::complex<double> o((double)ofs_all[q].first, (double)ofs_all[q].second);
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
      if (u >= 2 * p) return (u - 2 * p == v) ? 1.0 : 0.0;
      const std::complex<double> cv = C[(size_t)(u / 2) * p + v / 2];
      if ((u & 1) == 0) return (v & 1) ? -cv.imag() : cv.real();
      return (v & 1) ? cv.real() : cv.imag();
    };
    auto put = [&](int u, int v, double val) {
      unsigned char *row = B.data() + (size_t)q * M2L_BBYTES + (size_t)u * 128;
      if (T.kind == 0) {
        const int ch = v / 4, e = v % 4;
        const float f = tf32_round_host_m2l(val);
        std::memcpy(row + ((ch ^ (u & 7)) * 16) + 4 * e, &f, 4);
      } else {
        const int ch = v / 8, e = v % 8;
        const uint16_t b = bf16_round_host(val);
        std::memcpy(row + ((ch ^ (u & 7)) * 16) + 2 * e, &b, 2);
      }
    };
    for (int nn = 0; nn < p; ++nn)
      for (int k = 0; k < p; ++k) {
        const std::complex<double> cv = C[(size_t)nn * p + k];
        put(2 * nn, 2 * k, cv.real());
        put(2 * nn, 2 * k + 1, -cv.imag());
        put(2 * nn + 1, 2 * k, cv.imag());
        put(2 * nn + 1, 2 * k + 1, cv.real());
      }
    put(2 * p, 0, 1.0);
    put(2 * p + 1, 1, 1.0);
    // split columns: residual inputs meet the rounded column, rounded inputs the column residual
    for (int j = 0; j < T.nsplit; ++j)
      for (int u = 0; u < 2 * p + 2; ++u)
        for (int e = 0; e < 2; ++e) {
          const double full = Breal(u, 2 * j + e);
          const double hi = T.kind == 0 ? (double)tf32_round_host_m2l(full) : bf16_value(bf16_round_host(full));
          put(u, 2 * p + 4 * j + e, full);
          put(u, 2 * p + 4 * j + 2 + e, full - hi);
        }
  }
  // images and tiles
  int64_t rows = 0;
  std::vector<int4> tiles;
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
    for (int c = 0; c < 4; ++c)
      for (int f0 = fs; f0 <= fe; f0 += 128) tiles.push_back(make_int4(l, c, f0, 0));
  }
  T.rows_per_rhs = rows;
  T.ntiles = (int)tiles.size();
  T.stage_bytes = (M2L_WBYTES + maxcnt * M2L_BBYTES + 1023) & ~1023;
  T.smem = M2L_NSTG * T.stage_bytes + 1024;
  int maxsm = 0;
  FMMPC_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0));
  if (T.smem + 2048 > maxsm) throw Error(FMMPC_ERR_UNSUPPORTED, "tensor-core M2L: offset groups too large");
  T.img = H.pool.get<unsigned char>((size_t)H.nrhs_max * rows * 128);
  FMMPC_CUDA(cudaMemsetAsync(T.img, 0, (size_t)H.nrhs_max * rows * 128, H.stream));
  T.bmat = H.pool.get<unsigned char>(B.size());
  T.tiles = H.pool.get<int4>(tiles.size());
  T.groups = H.pool.get<int4>(groups.size());
  T.dxs = H.pool.get<int>(dxs.size());
  T.err = H.pool.get<int>(1);
  FMMPC_CUDA(cudaMemcpyAsync(T.bmat, B.data(), B.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemcpyAsync(T.dxs, dxs.data(), sizeof(int) * dxs.size(), cudaMemcpyHostToDevice, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(T.err, 0, sizeof(int), H.stream));
  FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
  FMMPC_CUDA(cudaFuncSetAttribute(k_m2l_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, T.smem));
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
  for (int c = 0; c < 4; ++c) {
    a.ngroups[c] = T.ngroups[c];
    a.goff[c] = T.goff[c];
    a.ooff[c] = T.ooff[c];
    a.nofs[c] = (c < 3 ? T.ooff[c + 1] : T.nofs_total) - T.ooff[c];
  }
  a.p = g.p;
  a.n = g.n;
  a.stage_bytes = T.stage_bytes;
  a.nsplit = T.nsplit;
  a.nks = T.kind == 0 ? (2 * g.p + 4 * T.nsplit + 7) / 8 : (2 * g.p + 4 * T.nsplit + 15) / 16;
  const int64_t lo = level_offset(2), hi = level_offset(g.L + 1);
  const int64_t threads = std::max<int64_t>((int64_t)nrhs * (hi - lo) * 8, (int64_t)nrhs * lo * g.p);
  const cpx<float> *M = (const cpx<float> *)Mv;
  if (T.kind == 0) k_m2l_pack<0><<<nblk(threads), 256, 0, s>>>(a, nrhs, lo, hi, M);
  else k_m2l_pack<1><<<nblk(threads), 256, 0, s>>>(a, nrhs, lo, hi, M);
  FMMPC_LAUNCH_CHECK();
  dim3 grid((unsigned)T.ntiles, (unsigned)nrhs);
  if (T.kind == 0) k_m2l_tc<0><<<grid, M2L_THREADS, T.smem, s>>>(a);
  else k_m2l_tc<1><<<grid, M2L_THREADS, T.smem, s>>>(a);
  FMMPC_LAUNCH_CHECK();
  return 2;
}

}  // namespace fmmpc
