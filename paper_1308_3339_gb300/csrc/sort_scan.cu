// Device-wide exclusive scan and a stable LSD radix sort (8-bit digits), used to order
// the grid nodes by Morton key (Sec. 5.1 tree construction) and to put the interaction
// lists of the dual tree traversal (Sec. 5.2) in canonical (level, target, source) order.
#include "common.cuh"

namespace fmmpc {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of the values of a 1024-thread block; returns the block total.
__device__ int32_t block_exclusive_scan(int32_t v, int32_t &excl) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t t = warp_tot[lane];
    int32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_tot[lane] = s - t;
    if (lane == 31) total = s;
  }
  __syncthreads();
  excl = warp_tot[wid] + x - v;
  int32_t tot = total;
  __syncthreads();  // warp_tot and total are reused by the next call
  return tot;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    if (k < n) s += in[k];
  }
  int32_t ex;
  int32_t tot = block_exclusive_scan(s, ex);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block scans the block sums in chunks, carrying the running total.
__global__ void k_scan_bsums(int32_t *__restrict__ bsum, int64_t nb, int32_t *__restrict__ total) {
  int32_t carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += SCAN_THREADS) {
    int64_t k = c0 + threadIdx.x;
    int32_t v = (k < nb) ? bsum[k] : 0;
    int32_t ex;
    int32_t tot = block_exclusive_scan(v, ex);
    if (k < nb) bsum[k] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_down(const int32_t *__restrict__ in, int64_t n, const int32_t *__restrict__ bsum,
                            int32_t *__restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t v[SCAN_ITEMS];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    v[i] = (k < n) ? in[k] : 0;
    s += v[i];
  }
  int32_t ex;
  block_exclusive_scan(s, ex);
  int32_t run = bsum[blockIdx.x] + ex;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    if (k < n) out[k] = run;
    run += v[i];
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_WARPS = 8;           // warps per block
constexpr int RS_ITEMS = 64;          // chunks of 32 per warp tile
constexpr int RS_TILE = 32 * RS_ITEMS;  // elements per warp tile

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int64_t ntiles,
                             int32_t *__restrict__ counts) {
  __shared__ int32_t h[RS_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * RS_WARPS + w;
  for (int d = lane; d < 256; d += 32) h[w][d] = 0;
  __syncwarp();
  if (tile < ntiles) {
    const int64_t base = tile * RS_TILE;
    for (int c = 0; c < RS_ITEMS; ++c) {
      int64_t k = base + c * 32 + lane;
      if (k < n) atomicAdd(&h[w][(keys[k] >> shift) & 0xff], 1);
    }
    __syncwarp();
    for (int d = lane; d < 256; d += 32) counts[(int64_t)d * ntiles + tile] = h[w][d];
  }
}

__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                int shift, int64_t ntiles, const int32_t *__restrict__ offs) {
  __shared__ int32_t o[RS_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * RS_WARPS + w;
  if (tile >= ntiles) return;  // whole warp leaves together
  for (int d = lane; d < 256; d += 32) o[w][d] = offs[(int64_t)d * ntiles + tile];
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = tile * RS_TILE;
  for (int c = 0; c < RS_ITEMS; ++c) {
    int64_t k = base + c * 32 + lane;
    bool valid = k < n;
    uint64_t key = valid ? kin[k] : 0;
    int d = valid ? (int)((key >> shift) & 0xff) : 256;  // 256 never equals a real digit
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt);
    int pos = valid ? o[w][d] + rank : 0;
    __syncwarp();
    if (valid) {
      kout[pos] = key;
      vout[pos] = vin[k];
      if (rank == 0) o[w][d] += __popc(peers);
    }
    __syncwarp();
  }
}

}  // namespace

void scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_host,
                        cudaStream_t s, DevPool &tmp) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  int32_t *bsum = tmp.get<int32_t>(nb + 1);
  int32_t *tot = tmp.get<int32_t>(1);
  k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
  FMMPC_LAUNCH_CHECK();
  k_scan_bsums<<<1, SCAN_THREADS, 0, s>>>(bsum, nb, tot);
  FMMPC_LAUNCH_CHECK();
  k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out);
  FMMPC_LAUNCH_CHECK();
  if (total_host) {
    FMMPC_CUDA(cudaMemcpyAsync(total_host, tot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FMMPC_CUDA(cudaStreamSynchronize(s));
  }
}

void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t s,
                    DevPool &tmp) {
  if (n <= 1) return;
  require(n < (int64_t(1) << 31), "radix sort: too many elements");
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  uint64_t *k2 = tmp.get<uint64_t>(n);
  uint32_t *v2 = tmp.get<uint32_t>(n);
  int32_t *counts = tmp.get<int32_t>(256 * ntiles);
  int32_t *offs = tmp.get<int32_t>(256 * ntiles);
  const unsigned grid = (unsigned)((ntiles + RS_WARPS - 1) / RS_WARPS);
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  int passes = (key_bits + 7) / 8;
  for (int ps = 0; ps < passes; ++ps) {
    int shift = 8 * ps;
    k_radix_hist<<<grid, 32 * RS_WARPS, 0, s>>>(ka, n, shift, ntiles, counts);
    FMMPC_LAUNCH_CHECK();
    scan_exclusive_i32(counts, offs, 256 * ntiles, nullptr, s, tmp);
    k_radix_scatter<<<grid, 32 * RS_WARPS, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, offs);
    FMMPC_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    FMMPC_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    FMMPC_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace fmmpc
