// FP64 Krylov solvers around the preconditioner (Sec. 3.1): CG, and GMRES(m) / FGMRES(m)
// with right preconditioning A P^{-1} y = b, x = P^{-1} y (Sec. 3.1 notation).  Zero
// initial iterate by default and a relative-residual stop (Sec. 6).  Several right-hand
// sides run side by side, each with its own Krylov space; vectors are [nrhs][N] FP64.
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2), so each orthogonalisation is
// a fused multi-dot and a fused update.  The small Hessenberg least-squares problem (Givens
// rotations) and the convergence test run on the host in the host-driven loop, and on the
// device in the graph-resident solver (one CUDA graph with a device-side loop condition).
#include <algorithm>
#include <chrono>
#include <cmath>

#include "handle.cuh"

namespace fmmpc {

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1024;  // per rhs at most; partial sums reduced in a second kernel or the last block
constexpr int MAXJ = 64;         // largest Krylov basis handled by the fused kernels

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Blocks of a reduction grid: four per SM (enough loads in flight for the vector sweeps;
// every further warp adds its own FP64 cross-lane sums, and FP64 issue is the scarce
// resource of these kernels on this GPU).
int red_blocks() {
  int dev = 0, nsm = 0;
  FMMPC_CUDA(cudaGetDevice(&dev));
  FMMPC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  return std::min(std::max(4 * nsm, 1), RED_BLOCKS);
}

// The operator A of the solves (fmmpc_set_operator), zero Dirichlet values outside the
// n x n block: 0 the five-point stencil (1/h^2)(4 u - neighbours) of Eq. e:axb; 1 the
// five-point flux form of -div(a grad u) (Sec. 4.4, Sec. 6.4), the coefficient of a face
// the mean of a at its two nodes, a at the (n+2)^2 nodes of the full grid; 2 the Q1
// stiffness of -lap (Sec. 6.1), 8/3 on the diagonal and -1/3 for the eight neighbours.
struct OpDev {
  int op, n;
  double s;          // 1/h^2
  const double *a;   // op 1: [(n+2)^2] coefficient
};

OpDev op_of(const fmmpc_handle &H) { return OpDev{H.op, H.g.n, 1.0 / (H.g.h * H.g.h), H.acoef}; }

__device__ __forceinline__ double op_at(const OpDev &o, const double *__restrict__ x, int64_t t) {
  const int n = o.n, lgn = __ffs(n) - 1;  // n is a power of two: shifts, not divisions
  const int64_t N = (int64_t)n * n;
  const int64_t k = t & (N - 1);
  const int i = (int)(k & (n - 1)), j = (int)(k >> lgn);
  if (o.op == 2) {
    double nb = 0.0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0) continue;
        const int ii = i + dx, jj = j + dy;
        if (ii >= 0 && ii < n && jj >= 0 && jj < n) nb += x[t + (int64_t)dy * n + dx];
      }
    return (8.0 / 3.0) * x[t] - (1.0 / 3.0) * nb;
  }
  if (o.op == 1) {
    const int W = n + 2;
    const int64_t I = (int64_t)(j + 1) * W + (i + 1);
    const double ac = o.a[I];
    const double aE = 0.5 * (ac + o.a[I + 1]), aW = 0.5 * (ac + o.a[I - 1]);
    const double aN = 0.5 * (ac + o.a[I + W]), aS = 0.5 * (ac + o.a[I - W]);
    double v = (aE + aW + aN + aS) * x[t];
    if (i > 0) v -= aW * x[t - 1];
    if (i < n - 1) v -= aE * x[t + 1];
    if (j > 0) v -= aS * x[t - n];
    if (j < n - 1) v -= aN * x[t + n];
    return o.s * v;
  }
  // five FP64 operations per node (three adds, one FMA, one product): the FP64 pipe, not
  // memory, bounds this stencil on this GPU
  const double xw = i > 0 ? x[t - 1] : 0.0, xe = i < n - 1 ? x[t + 1] : 0.0;
  const double xs = j > 0 ? x[t - n] : 0.0, xn = j < n - 1 ? x[t + n] : 0.0;
  return o.s * fma(4.0, x[t], -((xw + xe) + (xs + xn)));
}

__global__ void k_spmv5(OpDev o, int64_t total, const double *__restrict__ x, double *__restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) y[t] = op_at(o, x, t);
}

// Right-hand side of A u = b: op 0, b = f + g / h^2 at the stencil neighbours outside the
// interior block (Eq. e:pbound); op 1, the same with the face coefficient; op 2, the lumped
// Q1 load b = h^2 f (boundary data is rejected on the host for op 2).
__global__ void k_fold_rhs(OpDev o, int64_t total, const double *__restrict__ f, const double *__restrict__ g,
                           double *__restrict__ b) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int n = o.n, lgn = __ffs(n) - 1;
  const double s = o.s;
  const int64_t N = (int64_t)n * n;
  const int64_t rhs = t >> (2 * lgn), k = t & (N - 1);
  const int i = (int)(k & (n - 1)), j = (int)(k >> lgn);
  if (o.op == 2) {
    b[t] = f[t] / s;
    return;
  }
  double v = f[t];
  if (g) {
    const double *gg = g + rhs * 4 * n;
    double fe = 1.0, fw = 1.0, fn = 1.0, fs = 1.0;  // face coefficients toward the boundary
    if (o.op == 1) {
      const int W = n + 2;
      const int64_t I = (int64_t)(j + 1) * W + (i + 1);
      fe = 0.5 * (o.a[I] + o.a[I + 1]);
      fw = 0.5 * (o.a[I] + o.a[I - 1]);
      fn = 0.5 * (o.a[I] + o.a[I + W]);
      fs = 0.5 * (o.a[I] + o.a[I - W]);
    }
    if (j == 0) v += s * fs * gg[i];
    if (i == n - 1) v += s * fe * gg[n + j];
    if (j == n - 1) v += s * fn * gg[2 * n + (n - 1 - i)];
    if (i == 0) v += s * fw * gg[3 * n + (n - 1 - j)];
  }
  b[t] = v;
}

// Solves with (1/6) tridiag(1, 4, 1) along every row (cols = 0) or column (cols = 1) of every
// right-hand side: dst = scale * src on the way (src may alias dst).  cp[k], iden[k]: the
// Thomas coefficients of the constant matrix, formed once on the host.
__global__ void k_mass_sweep(int n, int nrhs, int cols, double scale, const double *__restrict__ src,
                             double *__restrict__ dst, const double *__restrict__ cp,
                             const double *__restrict__ iden) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nrhs * n) return;
  const int64_t N = (int64_t)n * n;
  const int lgn = __ffs(n) - 1;
  const int64_t rhs = t >> lgn, line = t & (n - 1);
  const int64_t base = rhs * N + (cols ? line : line * n), st = cols ? n : 1;
  double y = 0.0;
  for (int k = 0; k < n; ++k) {
    y = (scale * src[base + k * st] - (1.0 / 6.0) * y) * iden[k];
    dst[base + k * st] = y;
  }
  for (int k = n - 2; k >= 0; --k) {
    y = dst[base + k * st] - cp[k] * y;
    dst[base + k * st] = y;
  }
}

// acc[q] += <V_{i0+q}, w> (q < 8, i0 + q < nv; with self, index nv is <w, w>) over this
// thread's share of the N elements of one right-hand side, two elements per load (N is even
// and every vector starts 16-byte aligned).  Vr and wr point at that right-hand side.
__device__ __forceinline__ void mdot_chunk(int64_t N, const double *__restrict__ Vr, int64_t vs,
                                           const double *__restrict__ wr, int i0, int nv, bool with_self,
                                           double (&acc)[8]) {
  const int64_t N2 = N >> 1;
  const double2 *w2 = reinterpret_cast<const double2 *>(wr);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N2; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 wk = w2[k];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (i0 + q < nv) {
        const double2 v = reinterpret_cast<const double2 *>(Vr + (int64_t)(i0 + q) * vs)[k];
        acc[q] = fma(v.x, wk.x, fma(v.y, wk.y, acc[q]));
      } else if (with_self && i0 + q == nv) {
        acc[q] = fma(wk.x, wk.x, fma(wk.y, wk.y, acc[q]));
      }
    }
  }
}

// w -= sum_{i < nv} c[i] V_i over this thread's share of one right-hand side (two elements
// per load); returns this share of |w|^2 after the update.
__device__ __forceinline__ double update_chunk(int64_t N, const double *__restrict__ Vr, int64_t vs,
                                               const double *__restrict__ c, int nv, double *__restrict__ wr) {
  const int64_t N2 = N >> 1;
  double2 *w2 = reinterpret_cast<double2 *>(wr);
  double sq = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N2; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = w2[k];
    for (int i = 0; i < nv; ++i) {
      const double2 b = reinterpret_cast<const double2 *>(Vr + (int64_t)i * vs)[k];
      v.x = fma(-c[i], b.x, v.x);
      v.y = fma(-c[i], b.y, v.y);
    }
    w2[k] = v;
    sq = fma(v.x, v.x, fma(v.y, v.y, sq));
  }
  return sq;
}

// Sums a[q], q < 8, over the warp; lane 4q ends with the total of a[q].  A transposing
// butterfly: in each of the first three steps a lane keeps half of its values and adds the
// partner's copy of that half (4 + 2 + 1 adds), then two plain steps sum over the four lanes
// that hold the same value -- 9 FP64 adds where eight separate trees take 40.
__device__ __forceinline__ double warp_sum8(const double (&a)[8]) {
  const int lane = threadIdx.x & 31;
  const bool u4 = (lane & 16) != 0, u3 = (lane & 8) != 0, u2 = (lane & 4) != 0;
  double b[4], c[2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    b[i] = (u4 ? a[4 + i] : a[i]) + __shfl_xor_sync(0xffffffffu, u4 ? a[i] : a[4 + i], 16);
#pragma unroll
  for (int i = 0; i < 2; ++i)
    c[i] = (u3 ? b[2 + i] : b[i]) + __shfl_xor_sync(0xffffffffu, u3 ? b[i] : b[2 + i], 8);
  double d = (u2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, u2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// The block's sums of acc[q], q < nq (nq <= 8, block-uniform), into red[q] (a fixed order:
// lanes by the butterfly, then warps in turn).  red must hold 8 x (warps + 1) doubles.
__device__ __forceinline__ void block_sum8(const double (&acc)[8], int nq, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nq == 1) {
    double v = acc[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[8 + wid * 8] = v;
  } else {
    const double v = warp_sum8(acc);
    if ((lane & 3) == 0 && (lane >> 2) < nq) red[8 + wid * 8 + (lane >> 2)] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double sum = 0.0;
    for (int q = 0; q < nw; ++q) sum += red[8 + q * 8 + threadIdx.x];
    red[threadIdx.x] = sum;
  }
  __syncthreads();
}

// Sum of the np block partials pp[0 .. np) by one warp, lane l taking l, l + 32, ...: the
// loads go out eight at a time (an unrolled, predicated batch) rather than one round trip
// per step, then a shuffle tree.  The order of the additions is fixed.
__device__ __forceinline__ double warp_sum_parts(const double *__restrict__ pp, int np) {
  const int lane = threadIdx.x & 31;
  double sacc = 0.0;
  for (int b0 = 0; b0 < np; b0 += 256) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int bb = b0 + lane + 32 * u;
      v[u] = bb < np ? __ldcg(pp + bb) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) sacc += v[u];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
  return sacc;
}

// partial[rhs][i][blk] = sum over a slice of <V_i[rhs], w[rhs]>, i in [0, nv); V_i at V + i*vs.
// Vectors are taken in register groups of 8.
__global__ void __launch_bounds__(RED_THREADS) k_mdot_partial(int64_t N, int nv, const double *__restrict__ V,
                                                              int64_t vs, const double *__restrict__ w,
                                                              double *__restrict__ part, int with_self) {
  __shared__ double red[8 * (RED_THREADS / 32 + 1)];
  const int rhs = blockIdx.y;
  const double *wr = w + (int64_t)rhs * N;
  const int nt = nv + (with_self ? 1 : 0);  // index nv: <w, w>
  for (int i0 = 0; i0 < nt; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    mdot_chunk(N, V + (int64_t)rhs * N, vs, wr, i0, nv, with_self != 0, acc);
    const int nq = min(8, nt - i0);
    block_sum8(acc, nq, red);
    if (threadIdx.x < nq) part[((int64_t)rhs * MAXJ + i0 + threadIdx.x) * gridDim.x + blockIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
}

// out[rhs][i] = sum_blk partial, i < nv; acc[rhs][i] += the same for i < nacc.  One warp
// per (rhs, i): lanes stride over the block partials, then a shuffle reduction.
__global__ void k_mdot_final(int nv, int nblocks, const double *__restrict__ part, double *__restrict__ out,
                             double *__restrict__ acc, int nacc) {
  const int rhs = blockIdx.x, lane = threadIdx.x & 31;
  const int i = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= nv) return;
  const double sacc = warp_sum_parts(part + ((int64_t)rhs * MAXJ + i) * nblocks, nblocks);
  if (lane == 0) {
    out[rhs * MAXJ + i] = sacc;
    if (acc && i < nacc) acc[rhs * MAXJ + i] += sacc;
  }
}

// w[rhs] -= sum_i c[rhs][i] V_i[rhs], and part[rhs][0][blk] = sum over a slice of the new w^2
__global__ void k_mupdate_sq(int64_t N, int nv, const double *__restrict__ V, int64_t vs,
                             const double *__restrict__ c, double *__restrict__ w, double *__restrict__ part) {
  __shared__ double red[RED_THREADS / 32];
  const int rhs = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double sq = update_chunk(N, V + (int64_t)rhs * N, vs, c + rhs * MAXJ, nv, w + (int64_t)rhs * N);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane == 0) red[wid] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) t += red[q];
    part[(int64_t)rhs * MAXJ * gridDim.x + blockIdx.x] = t;
  }
}

// w[rhs] -= sum_i c[rhs][i] V_i[rhs]
__global__ void k_mupdate(int64_t N, int nrhs, int nv, const double *__restrict__ V, int64_t vs,
                          const double *__restrict__ c, double *__restrict__ w) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int rhs = (int)(t >> (__ffsll(N) - 1));  // N = n^2, a power of two
  double v = w[t];
  for (int i = 0; i < nv; ++i) v = fma(-c[rhs * MAXJ + i], V[i * vs + t], v);
  w[t] = v;
}

// x[rhs] += sum_i y[rhs][i] Z_i[rhs]
__global__ void k_maxpy(int64_t N, int nrhs, int nv, const double *__restrict__ Z, int64_t vs,
                        const double *__restrict__ y, double *__restrict__ x) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int rhs = (int)(t >> (__ffsll(N) - 1));  // N = n^2, a power of two
  double v = x[t];
  for (int i = 0; i < nv; ++i) v = fma(y[rhs * MAXJ + i], Z[i * vs + t], v);
  x[t] = v;
}

// y[rhs] = a[rhs] * x[rhs]  (a read from device, a = 0 allowed)
__global__ void k_scale(int64_t N, int nrhs, const double *__restrict__ a, const double *__restrict__ x,
                        double *__restrict__ y) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  y[t] = a[t >> (__ffsll(N) - 1)] * x[t];
}

// x += y
__global__ void k_add(int64_t total, const double *__restrict__ y, double *__restrict__ x) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  x[t] += y[t];
}

// y = b - y
__global__ void k_resid(int64_t total, const double *__restrict__ b, double *__restrict__ y) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  y[t] = b[t] - y[t];
}

// x += a p ; r -= a q  (CG), a per rhs
__global__ void k_cg_xr(int64_t N, int nrhs, const double *__restrict__ a, const double *__restrict__ p,
                        const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const double al = a[t >> (__ffsll(N) - 1)];
  x[t] = fma(al, p[t], x[t]);
  r[t] = fma(-al, q[t], r[t]);
}

// p = z + beta p
__global__ void k_cg_p(int64_t N, int nrhs, const double *__restrict__ beta, const double *__restrict__ z,
                       double *__restrict__ p) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  p[t] = fma(beta[t >> (__ffsll(N) - 1)], p[t], z[t]);
}

}  // namespace

// c = M^{-1} r for the consistent Q1 mass matrix M = h^2 (M1 (x) M1) of the interior nodes:
// tridiagonal solves along every row, then every column (the preconditioner of the Q1
// operator acts on the finite-element function of the residual, Sec. 6.1).
void q1_mass_solve(fmmpc_handle &H, const double *r, double *c, int nrhs) {
  const int n = H.g.n;
  const double h = H.g.h;
  k_mass_sweep<<<nblk((int64_t)nrhs * n), 256, 0, H.stream>>>(n, nrhs, 0, 1.0 / (h * h), r, c, H.q1tab, H.q1tab + n);
  k_mass_sweep<<<nblk((int64_t)nrhs * n), 256, 0, H.stream>>>(n, nrhs, 1, 1.0, c, c, H.q1tab, H.q1tab + n);
  FMMPC_LAUNCH_CHECK();
}

// z = P^{-1} r; with the Q1 operator, P^{-1} M^{-1} r through scratch (which may alias r when
// r is not needed afterwards).  in_capture: the apply's kernels go into the stream being
// captured instead of its own graph.
void precond_op(fmmpc_handle &H, const double *r, double *z, double *scratch, int nrhs, bool in_capture) {
  if (H.op == 2) {
    q1_mass_solve(H, r, scratch, nrhs);
    r = scratch;
  }
  if (in_capture) apply_fmm_eager(H, PART_FULL, r, z, nrhs);
  else apply_fmm(H, PART_FULL, r, z, nrhs);
}

namespace {

struct Ctx {
  fmmpc_handle &H;
  int64_t N;
  int nrhs;
  cudaStream_t s;
};

void ensure_ws(fmmpc_handle &H, int64_t nvec, bool flexible) {
  KrylovWs &k = H.kw;
  const int64_t N = (int64_t)H.g.n * H.g.n * H.nrhs_max;
  if (k.cap_vecs >= nvec && (!flexible || k.Z)) return;
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
  clear_solve_graphs(H);  // they hold the old workspace addresses
  ++H.ws_gen;             // and so do batch graphs kept by another handle
  if (k.hbuf) cudaFreeHost(k.hbuf);
  H.kpool.release();
  k = KrylovWs{};
  k.V = H.kpool.get<double>((size_t)N * nvec);
  k.Z = H.kpool.get<double>((size_t)N * (nvec - 1));
  k.w = H.kpool.get<double>(N);
  k.t = H.kpool.get<double>(N);
  k.b = H.kpool.get<double>(N);
  k.r = H.kpool.get<double>(N);
  k.x = H.kpool.get<double>(N);
  k.fin = H.kpool.get<double>(N);
  k.zin = H.kpool.get<double>(N);
  k.gin = H.kpool.get<double>((size_t)4 * H.g.n * H.nrhs_max);
  const int nr = H.nrhs_max;
  k.g_ctl = H.kpool.get<int>(16);
  k.g_done = H.kpool.get<int>(nr);
  k.g_iters = H.kpool.get<int>(nr);
  k.g_H = H.kpool.get<double>((size_t)nr * (MAXJ + 1) * MAXJ);
  k.g_cs = H.kpool.get<double>((size_t)nr * MAXJ);
  k.g_sn = H.kpool.get<double>((size_t)nr * MAXJ);
  k.g_g = H.kpool.get<double>((size_t)nr * (MAXJ + 1));
  k.g_bn = H.kpool.get<double>(nr);
  k.g_rel = H.kpool.get<double>(nr);
  k.g_sc = H.kpool.get<double>(nr);
  k.g_rtol = H.kpool.get<double>(1);
  k.g_cnt = H.kpool.get<int>(nr + 1);  // per right-hand side, then one over all of them
  FMMPC_CUDA(cudaMemsetAsync(k.g_ctl, 0, sizeof(int) * 16, H.stream));
  FMMPC_CUDA(cudaMemsetAsync(k.g_cnt, 0, sizeof(int) * (nr + 1), H.stream));
  k.dots = H.kpool.get<double>((size_t)H.nrhs_max * MAXJ * 4);
  k.part = H.kpool.get<double>((size_t)H.nrhs_max * MAXJ * RED_BLOCKS);
  k.scal = H.kpool.get<double>((size_t)H.nrhs_max * MAXJ * 2);
  FMMPC_CUDA(cudaMallocHost(&k.hbuf, sizeof(double) * H.nrhs_max * MAXJ * 8));
  k.cap_vecs = nvec;
}

// dots[rhs][0..nv) = <V_i, w>; if acc, acc += dots
// with_self: out[rhs][nv] = <w, w> as well (not accumulated into acc)
void mdot(Ctx &c, int nv, const double *V, int64_t vs, const double *w, double *out, double *acc,
          bool with_self = false) {
  const int nb = red_blocks();
  k_mdot_partial<<<dim3(nb, c.nrhs), RED_THREADS, 0, c.s>>>(c.N, nv, V, vs, w, c.H.kw.part, with_self ? 1 : 0);
  const int nt = nv + (with_self ? 1 : 0);
  k_mdot_final<<<dim3(c.nrhs, (nt + 7) / 8), 256, 0, c.s>>>(nt, nb, c.H.kw.part, out, acc, nv);
  FMMPC_LAUNCH_CHECK();
}

// w -= V coef (nv vectors), then out[rhs][0] = ||w||^2
void update_sq(Ctx &c, int nv, const double *V, int64_t vs, const double *coef, double *w, double *out) {
  const int nb = red_blocks();
  k_mupdate_sq<<<dim3(nb, c.nrhs), RED_THREADS, 0, c.s>>>(c.N, nv, V, vs, coef, w, c.H.kw.part);
  k_mdot_final<<<dim3(c.nrhs, 1), 256, 0, c.s>>>(1, nb, c.H.kw.part, out, nullptr, 0);
  FMMPC_LAUNCH_CHECK();
}

void to_host(Ctx &c, const double *d, size_t count) {
  FMMPC_CUDA(cudaMemcpyAsync(c.H.kw.hbuf, d, sizeof(double) * count, cudaMemcpyDeviceToHost, c.s));
  FMMPC_CUDA(cudaStreamSynchronize(c.s));
}

void precond(Ctx &c, const double *in, double *out) { precond_op(c.H, in, out, c.H.kw.zin, c.nrhs, false); }

void residual(Ctx &c, const double *b, const double *x, double *r) {
  spmv5(c.H, x, r, c.nrhs);
  k_resid<<<nblk(c.N * c.nrhs), 256, 0, c.s>>>(c.N * c.nrhs, b, r);
  FMMPC_LAUNCH_CHECK();
}

// per-rhs norms of v (length nrhs on host, in out)
void norms(Ctx &c, const double *v, std::vector<double> &out) {
  double *d = c.H.kw.dots;
  mdot(c, 1, v, 0, v, d, nullptr);  // with vs = 0 each rhs dots its own slice with itself
  to_host(c, d, (size_t)c.nrhs * MAXJ);
  out.resize(c.nrhs);
  for (int r = 0; r < c.nrhs; ++r) out[r] = std::sqrt(std::max(0.0, c.H.kw.hbuf[r * MAXJ]));
}

int gmres(Ctx &c, bool flexible, int m, int maxit, double rtol, const double *b, double *x,
          fmmpc_solve_info &info) {
  fmmpc_handle &H = c.H;
  KrylovWs &K = H.kw;
  const int64_t N = c.N, NR = N * c.nrhs, vs = N * H.nrhs_max;
  const int nr = c.nrhs;
  std::vector<double> bn, beta;
  norms(c, b, bn);
  for (double &v : bn) if (v == 0.0) v = 1.0;
  std::vector<double> Hm((size_t)nr * (m + 1) * m), cs((size_t)nr * m), sn((size_t)nr * m),
      gg((size_t)nr * (m + 1)), y((size_t)nr * MAXJ), hcol((size_t)nr * MAXJ);
  std::vector<int> done(nr, 0), rhs_iters(nr, 0);
  int it = 0;
  int status = FMMPC_OK;
  double *hy = K.hbuf + (size_t)nr * MAXJ * 2;  // pinned staging for y / scalars
  for (;;) {
    residual(c, b, x, K.r);
    norms(c, K.r, beta);
    bool all = true;
    for (int r = 0; r < nr; ++r) {
      if (!std::isfinite(beta[r])) return FMMPC_ERR_NAN;
      done[r] = beta[r] / bn[r] <= rtol;
      all = all && done[r];
    }
    if (all || it >= maxit) break;
    for (int r = 0; r < nr; ++r) hy[r] = done[r] ? 0.0 : 1.0 / beta[r];
    FMMPC_CUDA(cudaMemcpyAsync(K.scal, hy, sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
    k_scale<<<nblk(NR), 256, 0, c.s>>>(N, nr, K.scal, K.r, K.V);
    std::fill(gg.begin(), gg.end(), 0.0);
    for (int r = 0; r < nr; ++r) gg[(size_t)r * (m + 1)] = done[r] ? 0.0 : beta[r];
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      double *vj = K.V + (int64_t)j * vs;
      double *zj = flexible ? K.Z + (int64_t)j * vs : K.t;
      precond(c, vj, zj);
      spmv5(H, zj, K.w, nr);
      // classical Gram-Schmidt, h = V^T w, w -= V h, with the DGKS test: a second pass only
      // where the first removed more than half of ||w||^2 (cancellation has then cost
      // orthogonality).  ||w||^2 before comes with the dots, after with the update.
      double *d1 = K.dots, *hsum = K.dots + (size_t)nr * MAXJ;
      double *hb = K.hbuf + (size_t)4 * nr * MAXJ;  // pinned: h, then <.,w> with ||w||^2, ||w||^2 after
      FMMPC_CUDA(cudaMemsetAsync(hsum, 0, sizeof(double) * nr * MAXJ, c.s));
      double *wsq = K.scal + (size_t)nr * MAXJ;  // device: ||w||^2 after, [rhs][MAXJ]
      mdot(c, j + 1, K.V, vs, K.w, d1, hsum, true);
      update_sq(c, j + 1, K.V, vs, d1, K.w, wsq);
      std::vector<double> hn(nr), wb(nr);
      auto fetch = [&]() {
        FMMPC_CUDA(cudaMemcpyAsync(hb, hsum, sizeof(double) * nr * MAXJ, cudaMemcpyDeviceToHost, c.s));
        FMMPC_CUDA(cudaMemcpyAsync(hb + (size_t)nr * MAXJ, d1, sizeof(double) * nr * MAXJ, cudaMemcpyDeviceToHost, c.s));
        FMMPC_CUDA(cudaMemcpyAsync(hb + (size_t)2 * nr * MAXJ, wsq, sizeof(double) * nr * MAXJ,
                                   cudaMemcpyDeviceToHost, c.s));
        FMMPC_CUDA(cudaStreamSynchronize(c.s));
      };
      fetch();
      bool reorth = false;
      for (int r = 0; r < nr; ++r) {
        wb[r] = hb[(size_t)nr * MAXJ + (size_t)r * MAXJ + (j + 1)];
        const double wa = hb[(size_t)2 * nr * MAXJ + (size_t)r * MAXJ];
        if (!done[r] && wa < 0.5 * wb[r]) reorth = true;
      }
      if (reorth) {
        mdot(c, j + 1, K.V, vs, K.w, d1, hsum);
        update_sq(c, j + 1, K.V, vs, d1, K.w, wsq);
        fetch();
      }
      for (int r = 0; r < nr; ++r) {
        for (int i = 0; i <= j; ++i) hcol[(size_t)r * MAXJ + i] = hb[(size_t)r * MAXJ + i];
        hn[r] = std::sqrt(std::max(0.0, hb[(size_t)2 * nr * MAXJ + (size_t)r * MAXJ]));
      }
      ++it;
      bool conv_all = true;
      for (int r = 0; r < nr; ++r) {
        double *Hr = &Hm[(size_t)r * (m + 1) * m];
        for (int i = 0; i <= j; ++i) Hr[i * m + j] = hcol[(size_t)r * MAXJ + i];
        Hr[(j + 1) * m + j] = hn[r];
        double *csr = &cs[(size_t)r * m], *snr = &sn[(size_t)r * m], *g = &gg[(size_t)r * (m + 1)];
        for (int i = 0; i < j; ++i) {
          double a = Hr[i * m + j], bb = Hr[(i + 1) * m + j];
          Hr[i * m + j] = csr[i] * a + snr[i] * bb;
          Hr[(i + 1) * m + j] = -snr[i] * a + csr[i] * bb;
        }
        double a = Hr[j * m + j], bb = Hr[(j + 1) * m + j], rr = std::hypot(a, bb);
        if (rr == 0.0) { csr[j] = 1.0; snr[j] = 0.0; }
        else { csr[j] = a / rr; snr[j] = bb / rr; }
        Hr[j * m + j] = rr;
        Hr[(j + 1) * m + j] = 0.0;
        g[j + 1] = -snr[j] * g[j];
        g[j] = csr[j] * g[j];
        const double est = std::fabs(g[j + 1]) / bn[r];
        if (!std::isfinite(est)) return FMMPC_ERR_NAN;
        if (!done[r]) rhs_iters[r] = it;
        const bool ok = done[r] || est <= rtol || hn[r] == 0.0;
        conv_all = conv_all && ok;
        hy[r] = (hn[r] > 0.0 && !done[r]) ? 1.0 / hn[r] : 0.0;
      }
      FMMPC_CUDA(cudaMemcpyAsync(K.scal, hy, sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
      k_scale<<<nblk(NR), 256, 0, c.s>>>(N, nr, K.scal, K.w, K.V + (int64_t)(j + 1) * vs);
      FMMPC_LAUNCH_CHECK();
      if (conv_all) { ++j; break; }
    }
    // back substitution, y per rhs, then x += sum y_i z_i
    std::fill(y.begin(), y.end(), 0.0);
    for (int r = 0; r < nr; ++r) {
      if (done[r]) continue;
      const double *Hr = &Hm[(size_t)r * (m + 1) * m];
      const double *g = &gg[(size_t)r * (m + 1)];
      for (int i = j - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int k = i + 1; k < j; ++k) sacc -= Hr[i * m + k] * y[(size_t)r * MAXJ + k];
        y[(size_t)r * MAXJ + i] = (Hr[i * m + i] != 0.0) ? sacc / Hr[i * m + i] : 0.0;
      }
    }
    std::copy(y.begin(), y.end(), hy);
    FMMPC_CUDA(cudaMemcpyAsync(K.scal, hy, sizeof(double) * nr * MAXJ, cudaMemcpyHostToDevice, c.s));
    if (flexible) {
      k_maxpy<<<nblk(NR), 256, 0, c.s>>>(N, nr, j, K.Z, vs, K.scal, x);
    } else {
      FMMPC_CUDA(cudaMemsetAsync(K.t, 0, sizeof(double) * NR, c.s));
      k_maxpy<<<nblk(NR), 256, 0, c.s>>>(N, nr, j, K.V, vs, K.scal, K.t);
      precond(c, K.t, K.w);
      k_add<<<nblk(NR), 256, 0, c.s>>>(NR, K.w, x);
    }
    FMMPC_LAUNCH_CHECK();
    FMMPC_CUDA(cudaStreamSynchronize(c.s));
  }
  residual(c, b, x, K.r);
  norms(c, K.r, beta);
  double worst = 0.0;
  for (int r = 0; r < nr; ++r) {
    const double rel = beta[r] / bn[r];
    if (!std::isfinite(rel)) status = FMMPC_ERR_NAN;
    worst = std::max(worst, rel);
  }
  if (status == FMMPC_OK && worst > rtol) status = FMMPC_ERR_NOT_CONVERGED;
  info.iters = 0;
  for (int r = 0; r < nr; ++r) info.iters = std::max(info.iters, rhs_iters[r]);
  info.rel_res = worst;
  return status;
}

int pcg(Ctx &c, int maxit, double rtol, const double *b, double *x, fmmpc_solve_info &info) {
  fmmpc_handle &H = c.H;
  KrylovWs &K = H.kw;
  const int64_t N = c.N, NR = N * c.nrhs;
  const int nr = c.nrhs;
  double *r = K.r, *z = K.w, *p = K.V, *q = K.t;
  double *hy = K.hbuf + (size_t)nr * MAXJ * 2;
  std::vector<double> bn, rn;
  norms(c, b, bn);
  for (double &v : bn) if (v == 0.0) v = 1.0;
  residual(c, b, x, r);
  precond(c, r, z);
  FMMPC_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * NR, cudaMemcpyDeviceToDevice, c.s));
  auto dotv = [&](const double *a, const double *bb, std::vector<double> &out) {
    mdot(c, 1, a, 0, bb, K.dots, nullptr);
    to_host(c, K.dots, (size_t)nr * MAXJ);
    out.resize(nr);
    for (int i = 0; i < nr; ++i) out[i] = K.hbuf[i * MAXJ];
  };
  std::vector<double> rz, pq, rz2;
  dotv(r, z, rz);
  norms(c, r, rn);
  std::vector<int> done(nr, 0), its(nr, 0);
  int it = 0;
  bool all = true;
  for (int i = 0; i < nr; ++i) { done[i] = rn[i] / bn[i] <= rtol; all = all && done[i]; }
  while (!all && it < maxit) {
    spmv5(H, p, q, nr);
    dotv(p, q, pq);
    for (int i = 0; i < nr; ++i) hy[i] = (done[i] || pq[i] == 0.0) ? 0.0 : rz[i] / pq[i];
    FMMPC_CUDA(cudaMemcpyAsync(K.scal, hy, sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
    k_cg_xr<<<nblk(NR), 256, 0, c.s>>>(N, nr, K.scal, p, q, x, r);
    FMMPC_LAUNCH_CHECK();
    ++it;
    norms(c, r, rn);
    all = true;
    for (int i = 0; i < nr; ++i) {
      if (!std::isfinite(rn[i])) return FMMPC_ERR_NAN;
      if (!done[i]) its[i] = it;
      done[i] = done[i] || rn[i] / bn[i] <= rtol;
      all = all && done[i];
    }
    if (all) break;
    precond(c, r, z);
    dotv(r, z, rz2);
    for (int i = 0; i < nr; ++i) {
      hy[i] = (done[i] || rz[i] == 0.0) ? 0.0 : rz2[i] / rz[i];
      rz[i] = rz2[i];
    }
    FMMPC_CUDA(cudaMemcpyAsync(K.scal, hy, sizeof(double) * nr, cudaMemcpyHostToDevice, c.s));
    k_cg_p<<<nblk(NR), 256, 0, c.s>>>(N, nr, K.scal, z, p);
    FMMPC_LAUNCH_CHECK();
  }
  residual(c, b, x, r);
  norms(c, r, rn);
  double worst = 0.0;
  int status = FMMPC_OK;
  for (int i = 0; i < nr; ++i) {
    const double rel = rn[i] / bn[i];
    if (!std::isfinite(rel)) status = FMMPC_ERR_NAN;
    worst = std::max(worst, rel);
  }
  if (status == FMMPC_OK && worst > rtol) status = FMMPC_ERR_NOT_CONVERGED;
  info.iters = 0;
  for (int i = 0; i < nr; ++i) info.iters = std::max(info.iters, its[i]);
  info.rel_res = worst;
  return status;
}

}  // namespace

void spmv5(fmmpc_handle &H, const double *x, double *y, int nrhs) {
  const int64_t total = (int64_t)H.g.n * H.g.n * nrhs;
  k_spmv5<<<nblk(total), 256, 0, H.stream>>>(op_of(H), total, x, y);
  FMMPC_LAUNCH_CHECK();
}

int solve(fmmpc_handle &H, const double *f, const double *g, double *u, int nrhs,
          const fmmpc_solve_opts &o, fmmpc_solve_info &info) {
  require(o.method >= FMMPC_CG && o.method <= FMMPC_FGMRES, "unknown Krylov method");
  require(o.maxit >= 1 && o.rtol > 0.0, "maxit >= 1 and rtol > 0 required");
  const int m = (o.method == FMMPC_CG) ? 1 : std::min(o.restart, o.maxit);
  require(m >= 1 && m < MAXJ, "restart must be in [1, 63]");
  auto t0 = std::chrono::steady_clock::now();
  ensure_ws(H, o.method == FMMPC_CG ? 2 : m + 1, o.method == FMMPC_FGMRES);
  struct GraphsGuard {  // the solve's use_graphs option holds for this call only
    fmmpc_handle &H;
    bool saved;
    ~GraphsGuard() { H.graphs = saved; }
  } guard{H, H.graphs};
  require(o.use_graphs >= 0 && o.use_graphs <= 2, "use_graphs must be 0, 1 or 2");
  require(!(g && H.op == 2), "boundary data is not supported with the Q1 operator (its stencil needs the corners)");
  H.graphs = o.use_graphs == 1;
  Ctx c{H, (int64_t)H.g.n * H.g.n, nrhs, H.stream};
  const int64_t NR = c.N * nrhs;
  int st;
  if (o.use_graphs == 2) {
    st = solve_graphed(H, f, g, u, nrhs, o, info);  // one graph, device-side convergence
  } else {
    k_fold_rhs<<<nblk(NR), 256, 0, c.s>>>(op_of(H), NR, f, g, H.kw.b);
    FMMPC_LAUNCH_CHECK();
    if (o.method == FMMPC_CG) st = pcg(c, o.maxit, o.rtol, H.kw.b, u, info);
    else st = gmres(c, o.method == FMMPC_FGMRES, m, o.maxit, o.rtol, H.kw.b, u, info);
  }
  FMMPC_CUDA(cudaStreamSynchronize(c.s));
  info.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  info.t_setup_ms = H.t_setup_ms;
  info.status = st;
  return st;
}

}  // namespace fmmpc

// ====================================================================== batched solves
// Several independent problems (different grids) solved together by FGMRES(m), in
// lockstep: every Arnoldi step launches each active problem's preconditioner (a CUDA
// graph on that problem's stream, so the problems' applies overlap on the GPU), its SpMV
// and CGS2 kernels, and one host synchronisation serves the whole batch.  Converged
// problems drop out; each keeps its own Hessenberg system.
namespace fmmpc {

namespace {

struct BatchState {
  std::vector<double> Hm, cs, sn, g, y;
  double bn = 1.0, beta = 0.0;
  bool done = false, in_cycle = false;
  int j = 0, iters = 0, status = FMMPC_OK;
};

void sync_all(std::vector<fmmpc_handle *> &hs) {
  for (auto *h : hs) FMMPC_CUDA(cudaStreamSynchronize(h->stream));
}

// <v, v> of problem H into hbuf[slot] (asynchronous)
void norm2_async(fmmpc_handle &H, const double *v, double *dev_out, int slot) {
  Ctx c{H, (int64_t)H.g.n * H.g.n, 1, H.stream};
  mdot(c, 1, v, 0, v, dev_out, nullptr);
  FMMPC_CUDA(cudaMemcpyAsync(H.kw.hbuf + slot, dev_out, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
}

}  // namespace

int solve_batched(std::vector<fmmpc_handle *> &hs, const double *const *f, const double *const *gb,
                  double *const *u, const fmmpc_solve_opts &o, fmmpc_solve_info *infos) {
  require(o.method == FMMPC_FGMRES, "batched solve: FGMRES only");
  require(o.maxit >= 1 && o.rtol > 0.0, "maxit >= 1 and rtol > 0 required");
  const int m = std::min(o.restart, o.maxit);
  require(m >= 1 && m < MAXJ, "restart must be in [1, 63]");
  require(o.use_graphs >= 0 && o.use_graphs <= 2, "use_graphs must be 0, 1 or 2");
  const int np = (int)hs.size();
  auto t0 = std::chrono::steady_clock::now();
  if (o.use_graphs == 2) {
    const int rc = solve_batched_graphed(hs, f, gb, u, o, infos);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int p = 0; infos && p < np; ++p) infos[p].t_solve_ms = ms;
    return rc;
  }
  std::vector<BatchState> st(np);
  std::vector<bool> saved_graphs(np);
  for (int p = 0; p < np; ++p) {
    fmmpc_handle &H = *hs[p];
    saved_graphs[p] = H.graphs;
    H.graphs = o.use_graphs != 0;
    ensure_ws(H, m + 1, true);
    const int64_t N = (int64_t)H.g.n * H.g.n;
    require(!(gb && gb[p]) || H.op != 2, "boundary data is not supported with the Q1 operator");
    k_fold_rhs<<<nblk(N), 256, 0, H.stream>>>(op_of(H), N, f[p], gb ? gb[p] : nullptr, H.kw.b);
    FMMPC_LAUNCH_CHECK();
    norm2_async(H, H.kw.b, H.kw.dots, 0);
    BatchState &s = st[p];
    s.Hm.assign((size_t)(m + 1) * m, 0.0);
    s.cs.assign(m, 0.0);
    s.sn.assign(m, 0.0);
    s.g.assign(m + 1, 0.0);
    s.y.assign(MAXJ, 0.0);
  }
  sync_all(hs);
  for (int p = 0; p < np; ++p) {
    st[p].bn = std::sqrt(std::max(0.0, hs[p]->kw.hbuf[0]));
    if (st[p].bn == 0.0) st[p].bn = 1.0;
  }
  for (;;) {
    // residuals of the problems still running
    for (int p = 0; p < np; ++p) {
      if (st[p].done) continue;
      fmmpc_handle &H = *hs[p];
      Ctx c{H, (int64_t)H.g.n * H.g.n, 1, H.stream};
      residual(c, H.kw.b, u[p], H.kw.r);
      norm2_async(H, H.kw.r, H.kw.dots, 0);
    }
    sync_all(hs);
    bool any = false;
    for (int p = 0; p < np; ++p) {
      BatchState &s = st[p];
      s.in_cycle = false;
      if (s.done) continue;
      fmmpc_handle &H = *hs[p];
      s.beta = std::sqrt(std::max(0.0, H.kw.hbuf[0]));
      if (!std::isfinite(s.beta)) { s.done = true; s.status = FMMPC_ERR_NAN; continue; }
      if (s.beta / s.bn <= o.rtol) { s.done = true; continue; }
      if (s.iters >= o.maxit) { s.done = true; s.status = FMMPC_ERR_NOT_CONVERGED; continue; }
      s.in_cycle = true;
      s.j = 0;
      any = true;
      std::fill(s.g.begin(), s.g.end(), 0.0);
      s.g[0] = s.beta;
      const int64_t N = (int64_t)H.g.n * H.g.n;
      double *hy = H.kw.hbuf + 2 * MAXJ;
      hy[0] = 1.0 / s.beta;
      FMMPC_CUDA(cudaMemcpyAsync(H.kw.scal, hy, sizeof(double), cudaMemcpyHostToDevice, H.stream));
      k_scale<<<nblk(N), 256, 0, H.stream>>>(N, 1, H.kw.scal, H.kw.r, H.kw.V);
      FMMPC_LAUNCH_CHECK();
    }
    if (!any) break;
    for (int jj = 0; jj < m; ++jj) {
      bool active = false;
      for (int p = 0; p < np; ++p) {
        BatchState &s = st[p];
        if (!s.in_cycle) continue;
        active = true;
        fmmpc_handle &H = *hs[p];
        const int64_t N = (int64_t)H.g.n * H.g.n, vs = N * H.nrhs_max;
        Ctx c{H, N, 1, H.stream};
        double *vj = H.kw.V + (int64_t)s.j * vs, *zj = H.kw.Z + (int64_t)s.j * vs;
        precond_op(H, vj, zj, H.kw.zin, 1, false);
        spmv5(H, zj, H.kw.w, 1);
        double *d1 = H.kw.dots, *hsum = H.kw.dots + MAXJ;
        FMMPC_CUDA(cudaMemsetAsync(hsum, 0, sizeof(double) * MAXJ, H.stream));
        for (int pass = 0; pass < 2; ++pass) {
          mdot(c, s.j + 1, H.kw.V, vs, H.kw.w, d1, hsum);
          k_mupdate<<<nblk(N), 256, 0, H.stream>>>(N, 1, s.j + 1, H.kw.V, vs, d1, H.kw.w);
        }
        FMMPC_LAUNCH_CHECK();
        FMMPC_CUDA(cudaMemcpyAsync(H.kw.hbuf + MAXJ, hsum, sizeof(double) * (s.j + 1), cudaMemcpyDeviceToHost, H.stream));
        norm2_async(H, H.kw.w, H.kw.scal + MAXJ, 0);
      }
      if (!active) break;
      sync_all(hs);
      for (int p = 0; p < np; ++p) {
        BatchState &s = st[p];
        if (!s.in_cycle) continue;
        fmmpc_handle &H = *hs[p];
        const int j = s.j;
        const double hn = std::sqrt(std::max(0.0, H.kw.hbuf[0]));
        double *Hr = s.Hm.data();
        for (int i = 0; i <= j; ++i) Hr[i * m + j] = H.kw.hbuf[MAXJ + i];
        Hr[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = Hr[i * m + j], b = Hr[(i + 1) * m + j];
          Hr[i * m + j] = s.cs[i] * a + s.sn[i] * b;
          Hr[(i + 1) * m + j] = -s.sn[i] * a + s.cs[i] * b;
        }
        const double a = Hr[j * m + j], b = Hr[(j + 1) * m + j], rr = std::hypot(a, b);
        if (rr == 0.0) { s.cs[j] = 1.0; s.sn[j] = 0.0; }
        else { s.cs[j] = a / rr; s.sn[j] = b / rr; }
        Hr[j * m + j] = rr;
        Hr[(j + 1) * m + j] = 0.0;
        s.g[j + 1] = -s.sn[j] * s.g[j];
        s.g[j] = s.cs[j] * s.g[j];
        ++s.iters;
        ++s.j;
        const double est = std::fabs(s.g[j + 1]) / s.bn;
        const bool stop = !std::isfinite(est) || est <= o.rtol || hn == 0.0 || s.iters >= o.maxit || s.j >= m;
        if (!stop) {
          const int64_t N = (int64_t)H.g.n * H.g.n, vs = N * H.nrhs_max;
          double *hy = H.kw.hbuf + 2 * MAXJ;
          hy[0] = 1.0 / hn;
          FMMPC_CUDA(cudaMemcpyAsync(H.kw.scal, hy, sizeof(double), cudaMemcpyHostToDevice, H.stream));
          k_scale<<<nblk(N), 256, 0, H.stream>>>(N, 1, H.kw.scal, H.kw.w, H.kw.V + (int64_t)s.j * vs);
          FMMPC_LAUNCH_CHECK();
        } else {
          // end of this problem's cycle: y from the triangular system, x += Z y
          s.in_cycle = false;
          std::fill(s.y.begin(), s.y.end(), 0.0);
          for (int i = s.j - 1; i >= 0; --i) {
            double acc = s.g[i];
            for (int k = i + 1; k < s.j; ++k) acc -= Hr[i * m + k] * s.y[k];
            s.y[i] = (Hr[i * m + i] != 0.0) ? acc / Hr[i * m + i] : 0.0;
          }
          const int64_t N = (int64_t)H.g.n * H.g.n, vs = N * H.nrhs_max;
          double *hy = H.kw.hbuf + 2 * MAXJ;
          std::copy(s.y.begin(), s.y.begin() + MAXJ, hy);
          FMMPC_CUDA(cudaMemcpyAsync(H.kw.scal, hy, sizeof(double) * MAXJ, cudaMemcpyHostToDevice, H.stream));
          k_maxpy<<<nblk(N), 256, 0, H.stream>>>(N, 1, s.j, H.kw.Z, vs, H.kw.scal, u[p]);
          FMMPC_LAUNCH_CHECK();
        }
      }
      // the host buffers are reused by the next step: finish the copies issued above
      sync_all(hs);
    }
  }
  // true residuals
  for (int p = 0; p < np; ++p) {
    fmmpc_handle &H = *hs[p];
    Ctx c{H, (int64_t)H.g.n * H.g.n, 1, H.stream};
    residual(c, H.kw.b, u[p], H.kw.r);
    norm2_async(H, H.kw.r, H.kw.dots, 0);
  }
  sync_all(hs);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = FMMPC_OK;
  for (int p = 0; p < np; ++p) {
    const double rel = std::sqrt(std::max(0.0, hs[p]->kw.hbuf[0])) / st[p].bn;
    int status = st[p].status;
    if (!std::isfinite(rel)) status = FMMPC_ERR_NAN;
    else if (status == FMMPC_OK && rel > o.rtol) status = FMMPC_ERR_NOT_CONVERGED;
    if (infos) {
      infos[p].iters = st[p].iters;
      infos[p].rel_res = rel;
      infos[p].t_setup_ms = hs[p]->t_setup_ms;
      infos[p].t_solve_ms = ms;
      infos[p].status = status;
    }
    if (status != FMMPC_OK && worst == FMMPC_OK) worst = status;
    hs[p]->graphs = saved_graphs[p];
  }
  return worst;
}

}  // namespace fmmpc

// ====================================================================== graph-resident solves
// The whole Krylov solve as one CUDA graph: set-up nodes, then a conditional WHILE node whose
// body is one Arnoldi step (FGMRES/GMRES) or one CG iteration, and final nodes that recompute
// the true residual.  The Hessenberg column, the Givens rotations, the residual estimate, the
// convergence decision and (at the end of a cycle) the back substitution run on the device
// in one small kernel, which also sets the conditions of the loop and of the end-of-cycle
// IF node, so no step waits for the host: the host launches the graph once and reads the
// report when it has finished.  Orthogonalisation is classical Gram-Schmidt applied twice
// (CGS2) at every step.  The loop is bounded: every pass counts one preconditioner
// application and the loop stops at maxit, on a NaN, or when every right-hand side meets
// rtol.  Vector indices that depend on the step (V_j, Z_j, the number of basis vectors) are
// read by the kernels from the device control block.
namespace fmmpc {

namespace {

// control block (ints)
enum {
  KC_J = 0,       // step index within the current cycle
  KC_IT = 1,      // preconditioner applications so far (the loop's bound)
  KC_CYC = 2,     // 1: this step ended the cycle
  KC_DONE = 3,    // 1: every right-hand side met rtol (true residual)
  KC_NAN = 4,     // 1: a NaN or Inf met in a residual
  KC_MAXIT = 5,   // cap on KC_IT (set by the host before each launch)
  KC_JCNT = 6,    // basis vectors of the cycle that just ended
  KC_CONT = 7,    // value given to the loop condition
  KC_COUNT = 8
};

// x[rhs] += sum_{i < ctl[KC_JCNT]} y[rhs][i] Z_i[rhs]
__global__ void k_gmaxpy(const int *__restrict__ ctl, int64_t N, int nrhs, const double *__restrict__ Z, int64_t vs,
                         const double *__restrict__ y, double *__restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int rhs = (int)(t >> (__ffsll(N) - 1)), nv = ctl[KC_JCNT];
  double v = x[t];
  for (int i = 0; i < nv; ++i) v = fma(y[rhs * MAXJ + i], Z[i * vs + t], v);
  x[t] = v;
}

// V_{ctl[KC_J]}[rhs] = sc[rhs] w[rhs], and the same into t2 (the next preconditioner input)
__global__ void k_gscale_col(const int *__restrict__ ctl, int64_t N, int nrhs, const double *__restrict__ sc,
                             const double *__restrict__ w, double *__restrict__ V, int64_t vs, double *__restrict__ t2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const double v = sc[t >> (__ffsll(N) - 1)] * w[t];
  V[(int64_t)ctl[KC_J] * vs + t] = v;
  if (t2) t2[t] = v;
}

// Last block of a reduction grid to arrive: returns true in every thread of that block
// (counter cnt reset to zero by it).  Partial sums written before the call are visible.
__device__ __forceinline__ bool last_block(int *cnt) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(cnt, 1) == (int)(gridDim.x - 1));
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// out[rhs][i] = sum over blocks of part[rhs][i][blk], i < nout, in a fixed order (the last
// block of the grid, warp per i); acc: 0 none, 1 hsum = out, 2 hsum += out.
__device__ __forceinline__ void reduce_parts(const double *__restrict__ part, int rhs, int nout, double *__restrict__ out,
                                             double *__restrict__ hsum, int acc) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < nout; i += blockDim.x >> 5) {
    const double sacc = warp_sum_parts(part + ((int64_t)rhs * MAXJ + i) * gridDim.x, (int)gridDim.x);
    if (lane == 0) {
      out[rhs * MAXJ + i] = sacc;
      if (acc == 1) hsum[rhs * MAXJ + i] = sacc;
      else if (acc == 2) hsum[rhs * MAXJ + i] += sacc;
    }
  }
}

// The first CGS pass fused with the operator: w = A x (and Z_j = x for FGMRES), then
// d[rhs][i] = <V_i[rhs], w[rhs]>, i <= ctl[KC_J], reduced by the last block (hsum = d).  The
// first group of eight vectors takes w as it is formed; later groups reread it (each thread
// its own elements).
__global__ void __launch_bounds__(RED_THREADS) k_gapdots(const int *__restrict__ ctl, OpDev o, int64_t N,
                                                         const double *__restrict__ x, double *__restrict__ w,
                                                         double *__restrict__ Zb, const double *__restrict__ V,
                                                         int64_t vs, double *__restrict__ part, int *__restrict__ cnt,
                                                         double *__restrict__ out, double *__restrict__ hsum) {
  __shared__ double red[8 * (RED_THREADS / 32 + 1)];
  const int rhs = blockIdx.y, j = ctl[KC_J], nv = j + 1;
  const int64_t N2 = N >> 1, base = (int64_t)rhs * N;
  double2 *w2 = reinterpret_cast<double2 *>(w + base);
  const double2 *x2 = reinterpret_cast<const double2 *>(x + base);
  double2 *z2 = Zb ? reinterpret_cast<double2 *>(Zb + (int64_t)j * vs + base) : nullptr;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N2; k += (int64_t)gridDim.x * blockDim.x) {
      double2 wk;
      if (i0 == 0) {
        wk.x = op_at(o, x, base + 2 * k);
        wk.y = op_at(o, x, base + 2 * k + 1);
        w2[k] = wk;
        if (z2) z2[k] = x2[k];
      } else {
        wk = w2[k];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q < nv) {
          const double2 v = reinterpret_cast<const double2 *>(V + (int64_t)(i0 + q) * vs + base)[k];
          acc[q] = fma(v.x, wk.x, fma(v.y, wk.y, acc[q]));
        }
    }
    const int nq = min(8, nv - i0);
    block_sum8(acc, nq, red);
    if (threadIdx.x < nq) part[((int64_t)rhs * MAXJ + i0 + threadIdx.x) * gridDim.x + blockIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
  if (last_block(cnt + rhs)) {
    reduce_parts(part, rhs, nv, out, hsum, 1);
    if (threadIdx.x == 0) cnt[rhs] = 0;
  }
}

// The middle of CGS2 in one pass: w -= sum_{i <= j} c[rhs][i] V_i (c the first pass's
// coefficients, in the order of update_chunk), then d[rhs][i] = <V_i, w> (hsum += d): one
// sweep over the basis from memory, the second pass's reads served by L1 and L2.
__global__ void __launch_bounds__(RED_THREADS) k_gupdots(const int *__restrict__ ctl, int64_t N, const double *__restrict__ V,
                                                         int64_t vs, const double *__restrict__ c, double *__restrict__ w,
                                                         double *__restrict__ part, int *__restrict__ cnt,
                                                         double *__restrict__ out, double *__restrict__ hsum) {
  __shared__ double red[8 * (RED_THREADS / 32 + 1)];
  const int rhs = blockIdx.y, nv = ctl[KC_J] + 1;
  const int64_t N2 = N >> 1, base = (int64_t)rhs * N;
  double2 *w2 = reinterpret_cast<double2 *>(w + base);
  const double *cr = c + rhs * MAXJ;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N2; k += (int64_t)gridDim.x * blockDim.x) {
      double2 wk = w2[k];
      if (i0 == 0) {
        for (int i = 0; i < nv; ++i) {
          const double2 b = reinterpret_cast<const double2 *>(V + (int64_t)i * vs + base)[k];
          wk.x = fma(-cr[i], b.x, wk.x);
          wk.y = fma(-cr[i], b.y, wk.y);
        }
        w2[k] = wk;
      }
      // the second pass rereads V_i, which the update just brought into L1
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q < nv) {
          const double2 v = reinterpret_cast<const double2 *>(V + (int64_t)(i0 + q) * vs + base)[k];
          acc[q] = fma(v.x, wk.x, fma(v.y, wk.y, acc[q]));
        }
    }
    const int nq = min(8, nv - i0);
    block_sum8(acc, nq, red);
    if (threadIdx.x < nq) part[((int64_t)rhs * MAXJ + i0 + threadIdx.x) * gridDim.x + blockIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
  if (last_block(cnt + rhs)) {
    reduce_parts(part, rhs, nv, out, hsum, 2);
    if (threadIdx.x == 0) cnt[rhs] = 0;
  }
}

// Per-right-hand-side state of the graph-resident (F)GMRES.
struct GmState {
  double *Hm;    // [nrhs][(MAXJ + 1) MAXJ], entry (i, j) at i MAXJ + j (rotated)
  double *cs, *sn;  // [nrhs][MAXJ]
  double *g;     // [nrhs][MAXJ + 1]
  double *bn;    // [nrhs] ||b|| (1 where b = 0)
  double *rel;   // [nrhs] final true relative residual
  double *sc;    // [nrhs] scale of the next basis vector (0 for a finished right-hand side)
  double *rtol;  // [1]
  int *done, *iters;  // [nrhs]
};

__global__ void k_ginit(int *__restrict__ ctl, GmState st, int nrhs, const double *__restrict__ dots) {
  const int r = threadIdx.x;
  if (r < nrhs) {
    const double b = sqrt(fmax(0.0, dots[r * MAXJ]));
    st.bn[r] = b > 0.0 ? b : 1.0;
    st.iters[r] = 0;
    st.done[r] = 0;
  }
  if (r == 0) {
    ctl[KC_J] = 0;
    ctl[KC_IT] = 0;
    ctl[KC_CYC] = 0;
    ctl[KC_DONE] = 0;
    ctl[KC_NAN] = 0;
    ctl[KC_JCNT] = 0;
  }
}

// Start of a cycle from the true residual r (|r|^2 in dots[rhs][0]): per right-hand side
// done = |r| / |b| <= rtol, g = (|r|, 0, ...), scale 1/|r| of V_0 (0 when done); j = 0.
__global__ void k_grestart(int *__restrict__ ctl, GmState st, int nrhs, const double *__restrict__ dots) {
  __shared__ int s_all, s_nan;
  const int r = threadIdx.x;
  if (r == 0) { s_all = 1; s_nan = 0; }
  __syncthreads();
  if (r < nrhs) {
    const double beta = sqrt(fmax(0.0, dots[r * MAXJ]));
    const double rtol = st.rtol[0];
    if (!isfinite(beta) || !isfinite(dots[r * MAXJ])) atomicOr(&s_nan, 1);
    const int d = (beta / st.bn[r] <= rtol) ? 1 : 0;
    st.done[r] = d;
    double *g = st.g + r * (MAXJ + 1);
    for (int i = 0; i <= MAXJ; ++i) g[i] = 0.0;
    g[0] = d ? 0.0 : beta;
    st.sc[r] = (d || beta == 0.0) ? 0.0 : 1.0 / beta;
    if (!d) atomicAnd(&s_all, 0);
  }
  __syncthreads();
  if (r == 0) {
    ctl[KC_J] = 0;
    ctl[KC_DONE] = s_all;
    ctl[KC_NAN] |= s_nan;
  }
}

// End of an Arnoldi step: Hessenberg column j from the CGS2 coefficients h (hsum) and
// |w| (wsq), the previous rotations, a new rotation, the residual estimate |g_{j+1}| / |b|,
// the scale of V_{j+1}; the cycle ends when every right-hand side is within rtol (or has
// a zero |w|), at j + 1 = m, at maxit, or on a NaN; then y from the triangular system.
// Sets the condition of the end-of-cycle IF node.  Run by all threads of one block (one
// thread per right-hand side, nrhs <= blockDim.x).
__device__ __forceinline__ void gtail_run(int *__restrict__ ctl, GmState st, int nrhs, int m,
                                          const double *__restrict__ hsum, const double *__restrict__ wsq,
                                          double *__restrict__ y, cudaGraphConditionalHandle if_end) {
  __shared__ int s_ok, s_nan, s_cyc;
  const int r = threadIdx.x;
  const int j = ctl[KC_J], it = ctl[KC_IT] + 1;
  if (r == 0) { s_ok = 1; s_nan = 0; }
  __syncthreads();
  if (r < nrhs) {
    double *Hr = st.Hm + (int64_t)r * (MAXJ + 1) * MAXJ;
    double *cs = st.cs + r * MAXJ, *sn = st.sn + r * MAXJ, *g = st.g + r * (MAXJ + 1);
    for (int i = 0; i <= j; ++i) Hr[i * MAXJ + j] = hsum[r * MAXJ + i];
    const double hn = sqrt(fmax(0.0, wsq[r * MAXJ]));
    Hr[(j + 1) * MAXJ + j] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = Hr[i * MAXJ + j], b = Hr[(i + 1) * MAXJ + j];
      Hr[i * MAXJ + j] = cs[i] * a + sn[i] * b;
      Hr[(i + 1) * MAXJ + j] = -sn[i] * a + cs[i] * b;
    }
    const double a = Hr[j * MAXJ + j], b = Hr[(j + 1) * MAXJ + j], rr = hypot(a, b);
    if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
    else { cs[j] = a / rr; sn[j] = b / rr; }
    Hr[j * MAXJ + j] = rr;
    Hr[(j + 1) * MAXJ + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double est = fabs(g[j + 1]) / st.bn[r];
    if (!isfinite(est)) atomicOr(&s_nan, 1);
    const int done = st.done[r];
    if (!done) st.iters[r] = it;
    const bool ok = done || est <= st.rtol[0] || hn == 0.0;
    if (!ok) atomicAnd(&s_ok, 0);
    st.sc[r] = (hn > 0.0 && !done) ? 1.0 / hn : 0.0;
  }
  __syncthreads();
  if (r == 0) {
    const int cyc = (s_ok || s_nan || j + 1 >= m || it >= ctl[KC_MAXIT]) ? 1 : 0;
    s_cyc = cyc;
    ctl[KC_IT] = it;
    ctl[KC_CYC] = cyc;
    ctl[KC_JCNT] = j + 1;
    ctl[KC_J] = j + 1;
    ctl[KC_NAN] |= s_nan;
    cudaGraphSetConditional(if_end, (unsigned)cyc);
  }
  __syncthreads();
  if (s_cyc && r < nrhs) {  // back substitution (zeros for a finished right-hand side)
    const double *Hr = st.Hm + (int64_t)r * (MAXJ + 1) * MAXJ;
    const double *g = st.g + r * (MAXJ + 1);
    double *yr = y + r * MAXJ;
    const int jn = j + 1;
    for (int i = 0; i < MAXJ; ++i) yr[i] = 0.0;
    if (!st.done[r])
      for (int i = jn - 1; i >= 0; --i) {
        double acc = g[i];
        for (int k = i + 1; k < jn; ++k) acc -= Hr[i * MAXJ + k] * yr[k];
        yr[i] = (Hr[i * MAXJ + i] != 0.0) ? acc / Hr[i * MAXJ + i] : 0.0;
      }
  }
}

// The second CGS update, w -= V c, with |w|^2 reduced by each right-hand side's last block;
// the last right-hand side to finish then runs the step's tail (gtail_run) in the same
// launch: one kernel boundary fewer per Arnoldi step.
__global__ void __launch_bounds__(RED_THREADS) k_gupdate_tail(int *__restrict__ ctl, int64_t N, const double *__restrict__ V,
                                                              int64_t vs, const double *__restrict__ c,
                                                              double *__restrict__ w, double *__restrict__ part,
                                                              int *__restrict__ cnt, double *__restrict__ wsq, GmState st,
                                                              int nrhs, int m, const double *__restrict__ hsum,
                                                              double *__restrict__ y, cudaGraphConditionalHandle if_end) {
  __shared__ double red[RED_THREADS / 32];
  __shared__ int s_fin;
  const int rhs = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nv = ctl[KC_J] + 1;
  double sq = update_chunk(N, V + (int64_t)rhs * N, vs, c + rhs * MAXJ, nv, w + (int64_t)rhs * N);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane == 0) red[wid] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) t += red[q];
    part[(int64_t)rhs * MAXJ * gridDim.x + blockIdx.x] = t;
  }
  if (!last_block(cnt + rhs)) return;
  reduce_parts(part, rhs, 1, wsq, nullptr, 0);
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt[rhs] = 0;
    __threadfence();
    s_fin = atomicAdd(cnt + nrhs, 1) == nrhs - 1;
    if (s_fin) cnt[nrhs] = 0;
  }
  __syncthreads();
  if (!s_fin) return;
  __threadfence();
  gtail_run(ctl, st, nrhs, m, hsum, wsq, y, if_end);
}

// Condition of the loop: continue while some right-hand side is above rtol, no NaN was met
// and fewer than maxit preconditioner applications ran.
__global__ void k_gcond(int *__restrict__ ctl, cudaGraphConditionalHandle loop) {
  const int cont = (!ctl[KC_DONE] && !ctl[KC_NAN] && ctl[KC_IT] < ctl[KC_MAXIT]) ? 1 : 0;
  ctl[KC_CONT] = cont;
  cudaGraphSetConditional(loop, (unsigned)cont);
}

// Final report: true relative residual per right-hand side.
__global__ void k_gfinal(GmState st, int nrhs, const double *__restrict__ dots) {
  const int r = threadIdx.x;
  if (r < nrhs) st.rel[r] = sqrt(fmax(0.0, dots[r * MAXJ])) / st.bn[r];
}

// ---- CG (Sec. 3.1) with per-right-hand-side masks: the iteration's kernels are the fused
// k_cgf_* below
__global__ void k_cg_init(int *__restrict__ ctl, GmState st, int nrhs, const double *__restrict__ dots) {
  const int r = threadIdx.x;
  __shared__ int s_all, s_nan;
  if (r == 0) { s_all = 1; s_nan = 0; }
  __syncthreads();
  if (r < nrhs) {
    const double rn = sqrt(fmax(0.0, dots[r * MAXJ]));
    if (!isfinite(dots[r * MAXJ])) atomicOr(&s_nan, 1);  // fmax(0, NaN) would hide it
    const int d = rn / st.bn[r] <= st.rtol[0];
    st.done[r] = d;
    if (!d) atomicAnd(&s_all, 0);
  }
  __syncthreads();
  if (r == 0) {
    ctl[KC_DONE] = s_all;
    ctl[KC_NAN] |= s_nan;
  }
}

// ---- fused CG steps: each vector pass carries its inner product, finished in the grid's last
// block per right-hand side (a fixed order of block partials), which also takes the scalar
// step that follows, so one CG iteration is four vector kernels and the preconditioner.

// The block's sum of v into part[rhs][0][blockIdx.x]; true in every thread of the grid's last
// block to arrive for this right-hand side, whose warp 0 then holds the total in `tot`.
__device__ __forceinline__ bool block_partial_last(double v, double *__restrict__ part, int rhs, int *cnt,
                                                   double &tot) {
  __shared__ double red[RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[(int64_t)rhs * MAXJ * gridDim.x + blockIdx.x] = t;
  }
  if (!last_block(cnt + rhs)) return false;
  if (threadIdx.x == 0) cnt[rhs] = 0;
  tot = 0.0;
  if (wid == 0) tot = warp_sum_parts(part + (int64_t)rhs * MAXJ * gridDim.x, (int)gridDim.x);
  return true;
}

// q = A p and <p, q>; then alpha = <r, z> / <p, q> (0 for a finished right-hand side)
__global__ void __launch_bounds__(RED_THREADS) k_cgf_apdot(OpDev o, int64_t N, GmState st, const double *__restrict__ p,
                                                         double *__restrict__ q, double *__restrict__ part, int *cnt,
                                                         double *__restrict__ pq, const double *__restrict__ rz_old) {
  const int rhs = blockIdx.y;
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)rhs * N + k;
    const double v = op_at(o, p, t);
    q[t] = v;
    acc = fma(p[t], v, acc);
  }
  double tot;
  if (block_partial_last(acc, part, rhs, cnt, tot) && threadIdx.x == 0) {
    pq[rhs * MAXJ] = tot;
    st.sc[rhs] = (st.done[rhs] || tot == 0.0) ? 0.0 : rz_old[rhs * MAXJ] / tot;
  }
}

// x += alpha p, r -= alpha q and |r|^2; the last right-hand side to finish then does the
// convergence test of every right-hand side (iteration counts, done flags, NaN) and sets
// the condition of the solve's WHILE loop: some right-hand side still runs, below maxit
__global__ void __launch_bounds__(RED_THREADS) k_cgf_xr(int *__restrict__ ctl, int64_t N, int nrhs, GmState st,
                                                      const double *__restrict__ p, const double *__restrict__ q,
                                                      double *__restrict__ x, double *__restrict__ r,
                                                      double *__restrict__ part, int *cnt, double *__restrict__ dots,
                                                      cudaGraphConditionalHandle loop) {
  __shared__ int s_fin, s_all, s_nan;
  const int rhs = blockIdx.y;
  const double al = st.sc[rhs];
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)rhs * N + k;
    x[t] = fma(al, p[t], x[t]);
    const double rv = fma(-al, q[t], r[t]);
    r[t] = rv;
    acc = fma(rv, rv, acc);
  }
  double tot;
  if (!block_partial_last(acc, part, rhs, cnt, tot)) return;
  if (threadIdx.x == 0) {
    dots[rhs * MAXJ] = tot;
    __threadfence();
    s_fin = atomicAdd(cnt + nrhs, 1) == nrhs - 1;
    if (s_fin) cnt[nrhs] = 0;
    s_all = 1;
    s_nan = 0;
  }
  __syncthreads();
  if (!s_fin) return;
  __threadfence();
  const int it = ctl[KC_IT] + 1;
  for (int rr = threadIdx.x; rr < nrhs; rr += blockDim.x) {
    const double rn = sqrt(fmax(0.0, __ldcg(dots + rr * MAXJ)));
    if (!isfinite(rn)) atomicOr(&s_nan, 1);
    if (!st.done[rr]) st.iters[rr] = it;
    const int d = st.done[rr] || rn / st.bn[rr] <= st.rtol[0];
    st.done[rr] = d;
    if (!d) atomicAnd(&s_all, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[KC_IT] = it;
    ctl[KC_DONE] = s_all;
    ctl[KC_NAN] |= s_nan;
    const int more = (!s_all && !s_nan && it < ctl[KC_MAXIT]) ? 1 : 0;
    ctl[KC_CONT] = more;
    cudaGraphSetConditional(loop, (unsigned)more);
  }
}

// <r, z>; then beta = <r, z> / <r, z>_old (0 for a finished right-hand side), rz_old = <r, z>
__global__ void __launch_bounds__(RED_THREADS) k_cgf_rz(int64_t N, GmState st, const double *__restrict__ r,
                                                      const double *__restrict__ z, double *__restrict__ part, int *cnt,
                                                      double *__restrict__ rz_old) {
  const int rhs = blockIdx.y;
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)rhs * N + k;
    acc = fma(r[t], z[t], acc);
  }
  double tot;
  if (block_partial_last(acc, part, rhs, cnt, tot) && threadIdx.x == 0) {
    const double o = rz_old[rhs * MAXJ];
    st.sc[rhs] = (st.done[rhs] || o == 0.0) ? 0.0 : tot / o;
    rz_old[rhs * MAXJ] = tot;
  }
}

// Captures the work fn() issues on H.stream into `graph` after the nodes deps (H.stream is
// the capture stream meanwhile; the preconditioner's internal streams join it by events)
// and returns the capture's last nodes, the dependencies of whatever follows.
template <typename F>
std::vector<cudaGraphNode_t> capture_into(fmmpc_handle &H, cudaStream_t cs, cudaGraph_t graph,
                                          const std::vector<cudaGraphNode_t> &deps, F &&fn) {
  cudaStream_t user = H.stream;
  const int timing = H.timing;
  H.stream = cs;
  H.timing = 0;
  std::vector<cudaGraphNode_t> out;
  FMMPC_CUDA(cudaStreamBeginCaptureToGraph(cs, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                           cudaStreamCaptureModeThreadLocal));
  try {
    fn();
    cudaStreamCaptureStatus st{};
    const cudaGraphNode_t *d = nullptr;
    size_t nd = 0;
    FMMPC_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &d, nullptr, &nd));
    out.assign(d, d + nd);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    H.stream = user;
    H.timing = timing;
    throw;
  }
  H.stream = user;
  H.timing = timing;
  cudaGraph_t g = nullptr;
  FMMPC_CUDA(cudaStreamEndCapture(cs, &g));
  return out;
}

cudaGraphNode_t add_conditional(cudaGraph_t parent, const std::vector<cudaGraphNode_t> &deps,
                                cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t *body) {
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t n = nullptr;
  FMMPC_CUDA(cudaGraphAddNode(&n, parent, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
  *body = p.conditional.phGraph_out[0];
  return n;
}

GmState gm_state(KrylovWs &K) {
  return GmState{K.g_H, K.g_cs, K.g_sn, K.g_g, K.g_bn, K.g_rel, K.g_sc, K.g_rtol, K.g_done, K.g_iters};
}

// norms |v[rhs]|^2 into dots[rhs][0] (captured)
void gnorm2(Ctx &c, const double *v) {
  const int nb = red_blocks();
  k_mdot_partial<<<dim3(nb, c.nrhs), RED_THREADS, 0, c.H.stream>>>(c.N, 1, v, 0, v, c.H.kw.part, 0);
  k_mdot_final<<<dim3(c.nrhs, 1), 256, 0, c.H.stream>>>(1, nb, c.H.kw.part, c.H.kw.dots, nullptr, 0);
  FMMPC_LAUNCH_CHECK();
}

// Builds one problem's chain [set-up] -> WHILE [step (-> IF cycle end)] -> [final] into
// graph G.  Solves A u = b for the handle's internal vectors: b is folded from K.fin
// (and K.gin), the iterate is K.x.
void build_chain(fmmpc_handle &H, cudaGraph_t G, int method, int m, int nrhs, bool has_g) {
  KrylovWs &K = H.kw;
  if (!H.cstream) {  // the capture stream of solve graphs, at the highest priority (see the apply's streams)
    int prio_low = 0, prio_high = 0;
    FMMPC_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    FMMPC_CUDA(cudaStreamCreateWithPriority(&H.cstream, cudaStreamNonBlocking, prio_high));
  }
  cudaStream_t cs = H.cstream;
  const int64_t N = (int64_t)H.g.n * H.g.n, NR = N * nrhs, vs = N * H.nrhs_max;
  const double s = 1.0 / (H.g.h * H.g.h);
  const bool flexible = method == FMMPC_FGMRES;
  GmState st = gm_state(K);
  int *ctl = K.g_ctl;
  cudaGraphConditionalHandle hloop;
  FMMPC_CUDA(cudaGraphConditionalHandleCreate(&hloop, G, 0, cudaGraphCondAssignDefault));
  Ctx c{H, N, nrhs, cs};
  const OpDev od = op_of(H);
  auto precond = [&](const double *in, double *out, double *scratch) {
    precond_op(H, in, out, scratch, nrhs, true);
  };
  auto residual_c = [&](const double *b, const double *x, double *r) {
    k_spmv5<<<nblk(NR), 256, 0, H.stream>>>(od, NR, x, r);
    k_resid<<<nblk(NR), 256, 0, H.stream>>>(NR, b, r);
    FMMPC_LAUNCH_CHECK();
  };
  // ---- set-up
  const std::vector<cudaGraphNode_t> none;
  auto f_init = capture_into(H, cs, G, none, [&] {
    c.s = H.stream;
    k_fold_rhs<<<nblk(NR), 256, 0, H.stream>>>(od, NR, K.fin, has_g ? K.gin : nullptr, K.b);
    gnorm2(c, K.b);
    k_ginit<<<1, 64, 0, H.stream>>>(ctl, st, nrhs, K.dots);
    residual_c(K.b, K.x, K.r);
    gnorm2(c, K.r);
    if (method == FMMPC_CG) {
      // the loop body starts with z = P^{-1} r; p = 0 and <r, z>_old = 0 make its first
      // beta 0, so that p = z
      k_cg_init<<<1, 64, 0, H.stream>>>(ctl, st, nrhs, K.dots);
      FMMPC_CUDA(cudaMemsetAsync(K.V, 0, sizeof(double) * NR, H.stream));
      FMMPC_CUDA(cudaMemsetAsync(K.dots + (size_t)nrhs * MAXJ, 0, sizeof(double) * nrhs * MAXJ, H.stream));
    } else {
      k_grestart<<<1, 64, 0, H.stream>>>(ctl, st, nrhs, K.dots);
      k_gscale_col<<<nblk(NR), 256, 0, H.stream>>>(ctl, N, nrhs, K.g_sc, K.r, K.V, vs, K.t);
    }
    k_gcond<<<1, 1, 0, H.stream>>>(ctl, hloop);
    FMMPC_LAUNCH_CHECK();
  });
  cudaGraph_t body = nullptr;
  cudaGraphNode_t n_loop = add_conditional(G, f_init, hloop, cudaGraphCondTypeWhile, &body);
  cudaGraphConditionalHandle hif{};
  if (method != FMMPC_CG) FMMPC_CUDA(cudaGraphConditionalHandleCreate(&hif, body, 0, 0));
  double *hsum = K.dots + (size_t)nrhs * MAXJ, *wsq = K.scal + (size_t)nrhs * MAXJ;
  std::vector<cudaGraphNode_t> f_step;
  cudaGraph_t ifb = nullptr;
  if (method == FMMPC_CG) {
    // p in V_0, q in t, z in w; <r, z> of the last iteration in the second dots block
    double *p = K.V, *q = K.t, *z = K.w, *rz_old = K.dots + (size_t)nrhs * MAXJ;
    double *pq = K.dots + (size_t)2 * nrhs * MAXJ;
    // one iteration, rotated so that the convergence test ends it and sets the loop's own
    // condition (no IF node): z = P^{-1} r, beta, p = z + beta p, q = A p with alpha, then
    // x, r and the test
    const dim3 rgrid((unsigned)red_blocks(), nrhs);
    f_step = capture_into(H, cs, body, none, [&] {
      c.s = H.stream;
      precond(K.r, z, K.zin);
      k_cgf_rz<<<rgrid, RED_THREADS, 0, H.stream>>>(N, st, K.r, z, K.part, K.g_cnt, rz_old);
      k_cg_p<<<nblk(NR), 256, 0, H.stream>>>(N, nrhs, K.g_sc, z, p);
      k_cgf_apdot<<<rgrid, RED_THREADS, 0, H.stream>>>(od, N, st, p, q, K.part, K.g_cnt, pq, rz_old);
      k_cgf_xr<<<rgrid, RED_THREADS, 0, H.stream>>>(ctl, N, nrhs, st, p, q, K.x, K.r, K.part, K.g_cnt, K.dots,
                                                     hloop);
      FMMPC_LAUNCH_CHECK();
    });
  } else {
    f_step = capture_into(H, cs, body, none, [&] {
      c.s = H.stream;
      precond(K.t, K.zin, K.t);  // K.t holds v_j (written with V_j by the previous step)
      // w = A z_j with the first CGS pass, the first update with the second pass, the second
      // update with |w|^2: three sweeps over the basis, each reduction finished in its grid's
      // last block (a grid of a few blocks per SM keeps enough loads in flight)
      const dim3 rgrid((unsigned)red_blocks(), nrhs);
      double *d2 = K.dots + (size_t)2 * nrhs * MAXJ;
      k_gapdots<<<rgrid, RED_THREADS, 0, H.stream>>>(ctl, od, N, K.zin, K.w, flexible ? K.Z : nullptr, K.V, vs,
                                                     K.part, K.g_cnt, K.dots, hsum);
      k_gupdots<<<rgrid, RED_THREADS, 0, H.stream>>>(ctl, N, K.V, vs, K.dots, K.w, K.part, K.g_cnt, d2, hsum);
      k_gupdate_tail<<<rgrid, RED_THREADS, 0, H.stream>>>(ctl, N, K.V, vs, d2, K.w, K.part, K.g_cnt, wsq, st, nrhs, m,
                                                            hsum, K.scal, hif);
      k_gscale_col<<<nblk(NR), 256, 0, H.stream>>>(ctl, N, nrhs, K.g_sc, K.w, K.V, vs, K.t);
      FMMPC_LAUNCH_CHECK();
    });
    cudaGraphNode_t n_if = add_conditional(body, f_step, hif, cudaGraphCondTypeIf, &ifb);
    capture_into(H, cs, ifb, none, [&] {
      c.s = H.stream;
      if (flexible) {
        k_gmaxpy<<<nblk(NR), 256, 0, H.stream>>>(ctl, N, nrhs, K.Z, vs, K.scal, K.x);
      } else {
        FMMPC_CUDA(cudaMemsetAsync(K.t, 0, sizeof(double) * NR, H.stream));
        k_gmaxpy<<<nblk(NR), 256, 0, H.stream>>>(ctl, N, nrhs, K.V, vs, K.scal, K.t);
        precond(K.t, K.w, K.t);
        k_add<<<nblk(NR), 256, 0, H.stream>>>(NR, K.w, K.x);
      }
      residual_c(K.b, K.x, K.r);
      gnorm2(c, K.r);
      k_grestart<<<1, 64, 0, H.stream>>>(ctl, st, nrhs, K.dots);
      k_gscale_col<<<nblk(NR), 256, 0, H.stream>>>(ctl, N, nrhs, K.g_sc, K.r, K.V, vs, K.t);
      FMMPC_LAUNCH_CHECK();
    });
    capture_into(H, cs, body, {n_if}, [&] {
      k_gcond<<<1, 1, 0, H.stream>>>(ctl, hloop);
      FMMPC_LAUNCH_CHECK();
    });
  }
  // ---- final: the true residual
  capture_into(H, cs, G, {n_loop}, [&] {
    c.s = H.stream;
    residual_c(K.b, K.x, K.r);
    gnorm2(c, K.r);
    k_gfinal<<<1, 64, 0, H.stream>>>(st, nrhs, K.dots);
    FMMPC_LAUNCH_CHECK();
  });
}

}  // namespace

void clear_solve_graphs(fmmpc_handle &H) {
  for (auto &e : H.sgraphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  H.sgraphs.clear();
}

// The graph of (method, m, nrhs, has_g) for the handles hs (one chain each, side by side in
// one graph), built and instantiated on first use and kept by the first handle.
cudaGraphExec_t solve_graph(std::vector<fmmpc_handle *> &hs, int method, int m, int nrhs, bool has_g) {
  fmmpc_handle &H0 = *hs[0];
  std::vector<uint64_t> gens;
  for (auto *h : hs) gens.push_back(h->ws_gen);
  for (auto it = H0.sgraphs.begin(); it != H0.sgraphs.end(); ++it)
    if (it->method == method && it->m == m && it->nrhs == nrhs && it->has_g == (int)has_g &&
        it->nprob == (int)hs.size()) {
      if (it->gens == gens) return it->exec;
      cudaGraphExecDestroy(it->exec);  // a member's workspace moved since it was built
      H0.sgraphs.erase(it);
      break;
    }
  cudaGraph_t G = nullptr;
  FMMPC_CUDA(cudaGraphCreate(&G, 0));
  try {
    for (auto *h : hs) build_chain(*h, G, method, m, nrhs, has_g);
  } catch (...) {
    cudaGraphDestroy(G);
    throw;
  }
  SolveGraph e{method, m, nrhs, (int)has_g, (int)hs.size(), nullptr, gens};
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, G, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(G);
  FMMPC_CUDA(ie);
  H0.sgraphs.push_back(e);
  return e.exec;
}

// Solve through the graph: inputs copied into the handle's vectors, one launch, the report
// read back once.
int solve_graphed(fmmpc_handle &H, const double *f, const double *g, double *u, int nrhs, const fmmpc_solve_opts &o,
                  fmmpc_solve_info &info) {
  const int m = (o.method == FMMPC_CG) ? 1 : std::min(o.restart, o.maxit);
  KrylovWs &K = H.kw;
  const int64_t N = (int64_t)H.g.n * H.g.n, NR = N * nrhs;
  std::vector<fmmpc_handle *> hs{&H};
  cudaGraphExec_t ex = solve_graph(hs, o.method, m, nrhs, g != nullptr);
  cudaStream_t s = H.stream;
  FMMPC_CUDA(cudaMemcpyAsync(K.fin, f, sizeof(double) * NR, cudaMemcpyDeviceToDevice, s));
  if (g) FMMPC_CUDA(cudaMemcpyAsync(K.gin, g, sizeof(double) * 4 * H.g.n * nrhs, cudaMemcpyDeviceToDevice, s));
  FMMPC_CUDA(cudaMemcpyAsync(K.x, u, sizeof(double) * NR, cudaMemcpyDeviceToDevice, s));
  int *hc = reinterpret_cast<int *>(K.hbuf);
  double *hp = K.hbuf + 8;
  hc[0] = o.maxit;
  hp[0] = o.rtol;
  FMMPC_CUDA(cudaMemcpyAsync(K.g_ctl + KC_MAXIT, hc, sizeof(int), cudaMemcpyHostToDevice, s));
  FMMPC_CUDA(cudaMemcpyAsync(K.g_rtol, hp, sizeof(double), cudaMemcpyHostToDevice, s));
  FMMPC_CUDA(cudaGraphLaunch(ex, s));
  FMMPC_CUDA(cudaMemcpyAsync(u, K.x, sizeof(double) * NR, cudaMemcpyDeviceToDevice, s));
  double *hrel = K.hbuf + 16;
  int *hit = reinterpret_cast<int *>(K.hbuf + 16 + MAXJ), *hctl = hit + MAXJ;
  FMMPC_CUDA(cudaMemcpyAsync(hrel, K.g_rel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaMemcpyAsync(hit, K.g_iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaMemcpyAsync(hctl, K.g_ctl, sizeof(int) * KC_COUNT, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaStreamSynchronize(s));
  double worst = 0.0;
  int status = FMMPC_OK;
  info.iters = 0;
  for (int r = 0; r < nrhs; ++r) {
    if (!std::isfinite(hrel[r])) status = FMMPC_ERR_NAN;
    worst = std::max(worst, hrel[r]);
    info.iters = std::max(info.iters, hit[r]);
  }
  if (hctl[KC_NAN]) status = FMMPC_ERR_NAN;
  if (status == FMMPC_OK && worst > o.rtol) status = FMMPC_ERR_NOT_CONVERGED;
  info.rel_res = worst;
  return status;
}

// Independent problems solved by one graph: one chain per problem side by side (each with
// its own WHILE loop, so a problem stops at its own convergence), launched once on the
// first problem's stream after every problem's inputs are in place.
int solve_batched_graphed(std::vector<fmmpc_handle *> &hs, const double *const *f, const double *const *gb,
                          double *const *u, const fmmpc_solve_opts &o, fmmpc_solve_info *infos) {
  const int m = std::min(o.restart, o.maxit);
  const int np = (int)hs.size();
  bool has_g = false;
  for (int p = 0; p < np && gb; ++p) has_g = has_g || gb[p] != nullptr;
  for (auto *h : hs) ensure_ws(*h, m + 1, true);
  cudaGraphExec_t ex = solve_graph(hs, FMMPC_FGMRES, m, 1, has_g);
  fmmpc_handle &H0 = *hs[0];
  cudaStream_t s0 = H0.stream;
  for (int p = 0; p < np; ++p) {
    fmmpc_handle &H = *hs[p];
    KrylovWs &K = H.kw;
    const int64_t N = (int64_t)H.g.n * H.g.n;
    FMMPC_CUDA(cudaMemcpyAsync(K.fin, f[p], sizeof(double) * N, cudaMemcpyDeviceToDevice, s0));
    if (has_g) {
      if (gb[p]) FMMPC_CUDA(cudaMemcpyAsync(K.gin, gb[p], sizeof(double) * 4 * H.g.n, cudaMemcpyDeviceToDevice, s0));
      else FMMPC_CUDA(cudaMemsetAsync(K.gin, 0, sizeof(double) * 4 * H.g.n, s0));
    }
    FMMPC_CUDA(cudaMemcpyAsync(K.x, u[p], sizeof(double) * N, cudaMemcpyDeviceToDevice, s0));
    int *hc = reinterpret_cast<int *>(K.hbuf);
    double *hp = K.hbuf + 8;
    hc[0] = o.maxit;
    hp[0] = o.rtol;
    FMMPC_CUDA(cudaMemcpyAsync(K.g_ctl + KC_MAXIT, hc, sizeof(int), cudaMemcpyHostToDevice, s0));
    FMMPC_CUDA(cudaMemcpyAsync(K.g_rtol, hp, sizeof(double), cudaMemcpyHostToDevice, s0));
  }
  FMMPC_CUDA(cudaGraphLaunch(ex, s0));
  for (int p = 0; p < np; ++p) {
    fmmpc_handle &H = *hs[p];
    KrylovWs &K = H.kw;
    const int64_t N = (int64_t)H.g.n * H.g.n;
    FMMPC_CUDA(cudaMemcpyAsync(u[p], K.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s0));
    FMMPC_CUDA(cudaMemcpyAsync(K.hbuf + 16, K.g_rel, sizeof(double), cudaMemcpyDeviceToHost, s0));
    FMMPC_CUDA(cudaMemcpyAsync(K.hbuf + 17, K.g_iters, sizeof(int), cudaMemcpyDeviceToHost, s0));
    FMMPC_CUDA(cudaMemcpyAsync(K.hbuf + 18, K.g_ctl, sizeof(int) * KC_COUNT, cudaMemcpyDeviceToHost, s0));
  }
  FMMPC_CUDA(cudaStreamSynchronize(s0));
  int worst = FMMPC_OK;
  for (int p = 0; p < np; ++p) {
    KrylovWs &K = hs[p]->kw;
    const double rel = K.hbuf[16];
    const int iters = *reinterpret_cast<int *>(K.hbuf + 17);
    const int *hctl = reinterpret_cast<int *>(K.hbuf + 18);
    int status = FMMPC_OK;
    if (!std::isfinite(rel) || hctl[KC_NAN]) status = FMMPC_ERR_NAN;
    else if (rel > o.rtol) status = FMMPC_ERR_NOT_CONVERGED;
    if (infos) {
      infos[p].iters = iters;
      infos[p].rel_res = rel;
      infos[p].t_setup_ms = hs[p]->t_setup_ms;
      infos[p].status = status;
    }
    if (status != FMMPC_OK && worst == FMMPC_OK) worst = status;
  }
  return worst;
}

}  // namespace fmmpc
