// Lattice near field (P2P, Sec. 5.1 Eq. e:volume_integral restricted to neighbouring leaves)
// on the tensor cores.
//
// On the uniform grid the kernel between a target node of leaf X and a source node of
// leaf X + o depends only on their offset, so for each stencil offset o the near field is
// a matrix product: D[leaf][t] += sum_k W[leaf + o][k] * B_o[t][k], B_o[t][k] = ln|d(t, k, o)|
// (node units, cell-mean value at d = 0), t, k the 64 nodes of an 8x8 leaf.  One CTA takes
// 128 consecutive target leaves of one leaf row (M = 128, N = 64, K = 64 per offset) and
// sweeps the 37 stencil offsets, accumulating in TMEM.  FP32 accuracy from TF32 inputs:
// each operand is split hi + lo (hi a TF32 number, lo = x - hi) and the product is taken as
// hi*hi + hi*lo + lo*hi (three MMAs; the lo*lo term is below FP32 rounding).
//
// Data: the weights of each padded leaf row are stored as 16 chunks of 4 FP32 values per
// leaf, leaves contiguous within a chunk, so the 134 leaves a tile needs from one row are
// 16 contiguous 2144-byte runs -- 1-D bulk copies straight into the canonical K-major
// layout, and a shift by ox leaves is a 16-byte shift of the descriptor start.  The B_o
// pairs (hi, lo) are precomputed in the same layout (32 KB per offset).  A producer thread
// streams rows and offsets into double buffers; one thread issues the MMAs; all four
// warps read TMEM and write the result.
#include <cmath>
#include <cstring>

#include "handle.cuh"
#include "tc.cuh"

namespace fmmpc {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

constexpr int TC_TILE = 128;       // target leaves per CTA
constexpr int TC_BYTES_B = 32768;  // one offset: hi + lo, 64 x 64 FP32 each
constexpr int TC_MAXROWS = 33;

struct TcArgs {
  const float *ahi, *alo;  // [nrhs][NLY][16][NLX][4]
  const float *bmat;       // [nofs][hi, lo][16][64][4]
  double *out;
  int *err;
  int n, R, NLX, NLY, NS, nrows, npass;
  int row_oy[TC_MAXROWS], row_q0[TC_MAXROWS], row_q1[TC_MAXROWS], row_ox0[TC_MAXROWS];
};

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Weight strips: node (i, j) -> leaf (X, Y) = (i/8 + R, j/8 + R), k = (j%8) 8 + i%8.
__global__ void k_tc_strips(int n, int R, int NLX, int NLY, double h2, int64_t total, const double *__restrict__ r,
                            float *__restrict__ ahi, float *__restrict__ alo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t N = (int64_t)n * n;
  const int64_t rhs = t / N, q = t - rhs * N;
  const int i = (int)(q % n), j = (int)(q / n);
  const int X = i / 8 + R, Y = j / 8 + R, k = (j % 8) * 8 + (i % 8);
  const int64_t idx = (((rhs * NLY + Y) * 16 + k / 4) * NLX + X) * 4 + (k % 4);
  const double w = h2 * r[t];
  const float hi = tf32_round((float)w);
  ahi[idx] = hi;
  alo[idx] = (float)(w - (double)hi);
}

__global__ void __launch_bounds__(128, 1) k_p2p_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full_s[2], empty_s[2], full_b[2], empty_b[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, used_s, used_b;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int SB = 16 * a.NS * 16;  // bytes of one strip (hi or lo)
  unsigned char *strips = smem;   // [2 buffers][hi, lo][SB]
  unsigned char *bm = smem + 4 * SB;  // [2 buffers][32 KB]
  const int lx0 = blockIdx.x * TC_TILE, ly = blockIdx.y, rhs = blockIdx.z;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&full_s[b], 1);
      tc::mbar_init(&empty_s[b], 1);
      tc::mbar_init(&full_b[b], 1);
      tc::mbar_init(&empty_b[b], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_init_fence();
    abort_flag = 0;
    used_s = 0;
    used_b = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const int64_t rhs_off = (int64_t)rhs * a.NLY * 16 * a.NLX * 4;
  int issued_s = 0, issued_b = 0;
  if (warp == 0 && lane == 0) {
    // producer: weight rows of the stencil, then the B pairs of that row's offsets
    int boff = 0;
    for (int r = 0; r < a.nrows && !abort_flag; ++r) {
      const int sb = r & 1;
      if (r >= 2 && !tc::mbar_wait(&empty_s[sb], ((r >> 1) - 1) & 1, &abort_flag)) break;
      tc::mbar_expect_tx(&full_s[sb], 2 * SB);
      const int64_t Y = ly + a.R + a.row_oy[r];
      for (int hl = 0; hl < 2; ++hl) {
        const float *src = (hl ? a.alo : a.ahi) + rhs_off;
        unsigned char *dst = strips + (sb * 2 + hl) * SB;
        for (int c = 0; c < 16; ++c)
          tc::bulk_g2s(dst + c * a.NS * 16, src + ((Y * 16 + c) * a.NLX + lx0) * 4, a.NS * 16, &full_s[sb]);
      }
      issued_s = r + 1;
      bool stop = false;
      for (int q = a.row_q0[r]; q < a.row_q1[r]; ++q) {
        const int bi = boff & 1;
        if (boff >= 2 && !tc::mbar_wait(&empty_b[bi], ((boff >> 1) - 1) & 1, &abort_flag)) { stop = true; break; }
        tc::mbar_expect_tx(&full_b[bi], TC_BYTES_B);
        tc::bulk_g2s(bm + bi * TC_BYTES_B, a.bmat + (int64_t)q * (TC_BYTES_B / 4), TC_BYTES_B, &full_b[bi]);
        issued_b = ++boff;
      }
      if (stop) break;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = tc::idesc_tf32(128, 64);
    int boff = 0;
    bool first = true, ok = true;
    for (int r = 0; r < a.nrows && ok; ++r) {
      const int sb = r & 1;
      if (!tc::mbar_wait(&full_s[sb], (r >> 1) & 1, &abort_flag)) { ok = false; break; }
      used_s = r + 1;
      tc::fence_after();
      const uint32_t sh = tc::smem_addr(strips + (sb * 2) * SB), sl = tc::smem_addr(strips + (sb * 2 + 1) * SB);
      for (int q = a.row_q0[r]; q < a.row_q1[r]; ++q) {
        const int bi = boff & 1;
        if (!tc::mbar_wait(&full_b[bi], (boff >> 1) & 1, &abort_flag)) { ok = false; break; }
        used_b = boff + 1;
        tc::fence_after();
        const int ox = a.row_ox0[r] + (q - a.row_q0[r]);
        const uint32_t bh = tc::smem_addr(bm + bi * TC_BYTES_B), bl = bh + TC_BYTES_B / 2;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const uint32_t aoff = (uint32_t)((2 * s * a.NS + a.R + ox) * 16);
          const uint64_t ahd = tc::desc_kmajor(sh + aoff, a.NS * 16, 128);
          const uint64_t bhd = tc::desc_kmajor(bh + s * 2048, 1024, 128);
          tc::mma_tf32(tmem, ahd, bhd, idesc, first ? 0u : 1u);
          first = false;
          if (a.npass == 3) {
            const uint64_t ald = tc::desc_kmajor(sl + aoff, a.NS * 16, 128);
            const uint64_t bld = tc::desc_kmajor(bl + s * 2048, 1024, 128);
            tc::mma_tf32(tmem, ahd, bld, idesc, 1u);
            tc::mma_tf32(tmem, ald, bhd, idesc, 1u);
          }
        }
        tc::commit(&empty_b[bi]);
        ++boff;
      }
      tc::commit(&empty_s[sb]);
    }
    if (!ok) {
      abort_flag = 1;
      atomicOr(a.err, 1);
    }
    tc::commit(&done);  // completes when every MMA issued above has finished
  }
  __syncwarp();
  const bool finished = tc::mbar_wait(&done, 0, nullptr);
  __syncwarp();
  tc::fence_after();
  if (finished && !abort_flag) {
    const int X = lx0 + 32 * warp + lane;
    double *o = a.out + (int64_t)rhs * a.n * a.n + (int64_t)(ly * 8) * a.n + X * 8;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int t = c0 + jj;
        o[(int64_t)(t / 8) * a.n + (t % 8)] = -(double)v[jj] / (2.0 * PI);
      }
    }
  } else if (!finished && lane == 0) {
    atomicOr(a.err, 2);
  }
  tc::fence_before();
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0) {
    // drain bulk copies that were issued but never consumed (bounded waits)
    for (int u = used_s; u < issued_s; ++u) tc::mbar_wait(&full_s[u & 1], (u >> 1) & 1, nullptr);
    for (int u = used_b; u < issued_b; ++u) tc::mbar_wait(&full_b[u & 1], (u >> 1) & 1, nullptr);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 64);
  }
}

float tf32_round_host(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x1000u;  // half of the lowest kept mantissa bit: round to nearest
    u &= 0xffffe000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

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
  H.tcp.npass = (H.prec == FMMPC_PREC_FP32) ? 3 : 1;
  const size_t strip_floats = (size_t)H.nrhs_max * NL * 16 * NL * 4;
  H.tcp.ahi = H.pool.get<float>(strip_floats);
  H.tcp.alo = H.pool.get<float>(strip_floats);
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.ahi, 0, sizeof(float) * strip_floats, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.alo, 0, sizeof(float) * strip_floats, H.stream));
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
    std::vector<float> B((size_t)nofs * (TC_BYTES_B / 4), 0.0f);
    for (int r = 0; r < H.tcp.nrows; ++r)
      for (int q = q0s[r]; q < q1s[r]; ++q) {
        const int ox = ox0s[r] + (q - q0s[r]), oy = oys[r];
        float *Bq = B.data() + (size_t)q * (TC_BYTES_B / 4);
        for (int t = 0; t < 64; ++t)
          for (int k = 0; k < 64; ++k) {
            const int dx = (t % 8) - (k % 8) - 8 * ox, dy = (t / 8) - (k / 8) - 8 * oy;
            double v = (dx == 0 && dy == 0) ? cself : 0.5 * std::log((double)dx * dx + (double)dy * dy);
            if (variant) v += g.lnh;
            const float hi = tf32_round_host(v);
            const size_t e = ((size_t)(k / 4) * 64 + t) * 4 + (k % 4);
            Bq[e] = hi;
            Bq[TC_BYTES_B / 8 + e] = (float)(v - (double)hi);
          }
      }
    float *dB = H.pool.get<float>(B.size());
    FMMPC_CUDA(cudaMemcpyAsync(dB, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice, H.stream));
    FMMPC_CUDA(cudaStreamSynchronize(H.stream));
    (variant ? H.tcp.bmat_lnh : H.tcp.bmat) = dB;
  }
  H.tcp.err = H.pool.get<int>(1);
  FMMPC_CUDA(cudaMemsetAsync(H.tcp.err, 0, sizeof(int), H.stream));
  const int smem = 4 * 16 * H.tcp.NS * 16 + 2 * TC_BYTES_B;
  FMMPC_CUDA(cudaFuncSetAttribute(k_p2p_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  H.tcp.smem = smem;
}

// out[...] = -near / (2 pi) on the tensor cores; r is the FP64 right-hand side.
int run_p2p_tc(fmmpc_handle &H, const double *r, bool with_lnh, double *out, int nrhs, cudaStream_t s) {
  const Geo &g = H.g;
  const int64_t total = (int64_t)g.n * g.n * nrhs;
  k_tc_strips<<<nblk(total), 256, 0, s>>>(g.n, g.R, H.tcp.NLX, H.tcp.NLY, g.h * g.h, total, r, H.tcp.ahi, H.tcp.alo);
  FMMPC_LAUNCH_CHECK();
  TcArgs a{};
  a.ahi = H.tcp.ahi;
  a.alo = H.tcp.alo;
  a.bmat = with_lnh ? H.tcp.bmat_lnh : H.tcp.bmat;
  a.out = out;
  a.err = H.tcp.err;
  a.n = g.n;
  a.R = g.R;
  a.NLX = H.tcp.NLX;
  a.NLY = H.tcp.NLY;
  a.NS = H.tcp.NS;
  a.nrows = H.tcp.nrows;
  a.npass = H.tcp.npass;
  for (int i = 0; i < a.nrows; ++i) {
    a.row_oy[i] = H.tcp.row_oy[i];
    a.row_q0[i] = H.tcp.row_q0[i];
    a.row_q1[i] = H.tcp.row_q1[i];
    a.row_ox0[i] = H.tcp.row_ox0[i];
  }
  dim3 grid((1 << g.L) / TC_TILE, 1 << g.L, nrhs);
  k_p2p_tc<<<grid, 128, H.tcp.smem, s>>>(a);
  FMMPC_LAUNCH_CHECK();
  return 2;
}

}  // namespace fmmpc
