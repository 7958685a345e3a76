// Boundary-element set-up (Sec. 4.3): constant elements, no nodes at the corners, 4n
// equal elements on the square, collocation at their midpoints.  The single-layer
// matrix S_mk = int_{Gamma_k} G(y_m, y) dGamma (left side of Eq. e:ubound) is assembled in
// FP64 from the closed-form element integral (Sec. 4.2).  The square's 90-degree rotation
// symmetry makes S block circulant over the four sides, so a 4-point DFT over the side
// index splits it into three n x n blocks (one complex); each is inverted once by
// Gauss-Jordan elimination with partial pivoting, and the apply works in that basis.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"

namespace fmmpc {

namespace {

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// along-side coordinate and signed normal offset (node units) of a point, per side
__device__ __forceinline__ void side_coords_d(int side, double np1, double x, double y, double &u, double &d) {
  switch (side) {
    case 0: u = x; d = -y; break;
    case 1: u = y; d = x - np1; break;
    case 2: u = np1 - x; d = y - np1; break;
    default: u = np1 - y; d = -x; break;
  }
}

__device__ __forceinline__ double seg_log_int_d(double s1, double ell, double d) {
  const double s2 = s1 + ell;
  const double A1 = s1 * s1 + d * d, A2 = s2 * s2 + d * d;
  double v = 0.5 * (ell * log(A2) + s1 * log1p(ell * (s1 + s2) / A1)) - ell;
  if (d != 0.0) v += d * atan2(ell * d, d * d + s1 * s2);
  return v;
}

// S_mk = -(h/2pi) (int_k ln|y_m - y|_node ds_node + l ln h)  (physical units)
__global__ void k_bem_S(int n, double h, double lnh, double *__restrict__ S) {
  const int NG = 4 * n;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)NG * NG) return;
  const int mrow = (int)(t / NG), k = (int)(t % NG);
  const double ell = (n + 1.0) / n, np1 = n + 1.0;
  // collocation point m in node units
  const int sm = mrow / n, km = mrow % n;
  const double tm = (km + 0.5) * ell;
  double x, y;
  switch (sm) {
    case 0: x = tm; y = 0; break;
    case 1: x = np1; y = tm; break;
    case 2: x = np1 - tm; y = np1; break;
    default: x = 0; y = np1 - tm; break;
  }
  const int sk = k / n, kk = k % n;
  double u, d;
  side_coords_d(sk, np1, x, y, u, d);
  double I;
  if (sk == sm) I = seg_log_int_d((kk - km - 0.5) * ell, ell, 0.0);  // same side: exact offsets
  else I = seg_log_int_d(kk * ell - u, ell, d);
  S[t] = -(h / (2.0 * PI)) * (I + ell * lnh);
}

// First block row of -1/2 I + K, K_mk = int_k dG/dn_y(y_m, y) dGamma = (1/2pi) atan2(l d,
// d^2 + s1 s2) with d the signed normal offset of y_m from element k's line (zero on the
// same side): the system (-1/2 I + K) mu = -(V r)|_Gamma of the double-layer correction.
__global__ void k_bem_Kdl(int n, double *__restrict__ A) {
  const int NG = 4 * n;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * NG) return;
  const int mrow = (int)(t / NG), k = (int)(t % NG);
  const double ell = (n + 1.0) / n, np1 = n + 1.0;
  const double x = (mrow + 0.5) * ell, y = 0.0;  // collocation point mrow of side 0
  const int sk = k / n, kk = k % n;
  double v = 0.0;
  if (sk == 0) {
    v = (k == mrow) ? -0.5 : 0.0;
  } else {
    double u, d;
    side_coords_d(sk, np1, x, y, u, d);
    const double s1 = kk * ell - u, s2 = s1 + ell;
    v = atan2(ell * d, d * d + s1 * s2) / (2.0 * PI);
  }
  A[t] = v;
}

__global__ void k_gj_pivot(int N, int k, const double *__restrict__ A, int *__restrict__ piv,
                           double *__restrict__ pinv, double *__restrict__ pabs) {
  __shared__ double best[1024];
  __shared__ int bi[1024];
  double b = -1.0;
  int ib = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    double v = fabs(A[(int64_t)i * N + k]);
    if (v > b) { b = v; ib = i; }
  }
  best[threadIdx.x] = b;
  bi[threadIdx.x] = ib;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = best[threadIdx.x + s];
      int oi = bi[threadIdx.x + s];
      if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bi[threadIdx.x])) {
        best[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    piv[k] = bi[0];
    const double pv = A[(int64_t)bi[0] * N + k];
    pabs[k] = fabs(pv);
    *pinv = (pv != 0.0) ? 1.0 / pv : 0.0;
  }
}

// swap rows k and piv[k]; row k <- row k / pivot with A[k][k] replaced by 1 first
__global__ void k_gj_swap_scale(int N, int k, double *__restrict__ A, const int *__restrict__ piv,
                                const double *__restrict__ pinv, double *__restrict__ col) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int p = piv[k];
  double a = A[(int64_t)k * N + j], b = A[(int64_t)p * N + j];
  if (p != k) A[(int64_t)p * N + j] = a;
  const double v = (j == k) ? 1.0 : b;
  A[(int64_t)k * N + j] = v * (*pinv);
  (void)col;
}

__global__ void k_gj_colsave(int N, int k, const double *__restrict__ A, double *__restrict__ col) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  col[i] = (i == k) ? 0.0 : A[(int64_t)i * N + k];
}

// rows i != k: A[i][j] = (j == k ? 0 : A[i][j]) - col[i] A[k][j]
__global__ void k_gj_elim(int N, int k, double *__restrict__ A, const double *__restrict__ col) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= N || i == k) return;
  const double f = col[i];
  if (f == 0.0 && j != k) return;
  double *row = A + (int64_t)i * N;
  const double base = (j == k) ? 0.0 : row[j];
  row[j] = base - f * A[(int64_t)k * N + j];
}

__global__ void k_swap_cols(int N, double *__restrict__ A, int c1, int c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double *row = A + (int64_t)i * N;
  double t = row[c1];
  row[c1] = row[c2];
  row[c2] = t;
}

// From the first block row of S (n x 4n): S^0 and S^2 (n x n) and the real form of S^1,
// E = [[S0 - S2, -(S1 - S3)], [S1 - S3, S0 - S2]] (2n x 2n).
__global__ void k_bem_blocks(int n, const double *__restrict__ S, double *__restrict__ B0, double *__restrict__ B2,
                             double *__restrict__ E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int64_t m = t / n;
  const int k = (int)(t % n);
  const double *row = S + m * 4 * n;
  const double s0 = row[k], s1 = row[n + k], s2 = row[2 * n + k], s3 = row[3 * n + k];
  B0[m * n + k] = (s0 + s2) + (s1 + s3);
  B2[m * n + k] = (s0 + s2) - (s1 + s3);
  const double re = s0 - s2, im = s1 - s3;
  E[m * 2 * n + k] = re;
  E[m * 2 * n + n + k] = -im;
  E[(m + n) * 2 * n + k] = im;
  E[(m + n) * 2 * n + n + k] = re;
}

// T[m] = [inv(S^0) | inv(S^2) | A | B][m] with A + i B = inv(S^1): A, B from the left
// column blocks of inv(E).
__global__ void k_bem_pack(int n, const double *__restrict__ B0, const double *__restrict__ B2,
                           const double *__restrict__ E, double *__restrict__ T) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int64_t m = t / n;
  const int k = (int)(t % n);
  double *o = T + m * 4 * n;
  o[k] = B0[m * n + k];
  o[n + k] = B2[m * n + k];
  o[2 * n + k] = E[m * 2 * n + k];
  o[3 * n + k] = E[(m + n) * 2 * n + k];
}

// In-place Gauss-Jordan inverse of the N x N matrix A (row-major, device) with partial
// pivoting; returns the smallest pivot magnitude (0 for a singular matrix).
double gj_invert(double *A, int N, cudaStream_t s, DevPool &tmp) {
  int *piv = tmp.get<int>(N);
  double *pinv = tmp.get<double>(1), *pabs = tmp.get<double>(N), *col = tmp.get<double>(N);
  for (int k = 0; k < N; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(N, k, A, piv, pinv, pabs);
    k_gj_swap_scale<<<nblk(N), 256, 0, s>>>(N, k, A, piv, pinv, col);
    k_gj_colsave<<<nblk(N), 256, 0, s>>>(N, k, A, col);
    k_gj_elim<<<dim3(nblk(N), N), 256, 0, s>>>(N, k, A, col);
  }
  FMMPC_LAUNCH_CHECK();
  std::vector<int> hp(N);
  std::vector<double> ha(N);
  FMMPC_CUDA(cudaMemcpyAsync(hp.data(), piv, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaMemcpyAsync(ha.data(), pabs, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaStreamSynchronize(s));
  double amin = ha[0];
  for (int k = 0; k < N; ++k) amin = std::min(amin, ha[k]);
  for (int k = N - 1; k >= 0; --k)
    if (hp[k] != k) k_swap_cols<<<nblk(N), 256, 0, s>>>(N, A, k, hp[k]);
  FMMPC_LAUNCH_CHECK();
  return amin;
}

}  // namespace

namespace {
// x = hi + lo, hi = fl32(x), lo = fl32(x - hi)
__global__ void k_split_f2(int64_t total, const double *__restrict__ x, float *__restrict__ hi, float *__restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const double v = x[t];
  const float h = (float)v;
  hi[t] = h;
  lo[t] = (float)(v - (double)h);
}
}  // namespace

void init_bem(fmmpc_handle &H, DevPool &tmp) {
  // S is block circulant in the four sides (the 90-degree rotation of the square maps
  // element (s, k) to (s+1, k)), so a 4-point DFT over the side index block-diagonalises
  // it: with S_d = S[(0, .), (d, .)], S^0 = S0+S1+S2+S3, S^2 = S0-S1+S2-S3 (real) and
  // S^1 = (S0 - S2) + i (S1 - S3).  The apply needs exactly the inverses of these blocks,
  // [inv(S^0) | inv(S^2) | Re inv(S^1) | Im inv(S^1)] per row, so only the first block row
  // of S is assembled and three n x n systems are inverted (the complex one through its
  // 2n x 2n real form [[Re, -Im], [Im, Re]], whose inverse is [[A, -B], [B, A]]).
  const Geo &g = H.g;
  const int n = g.n, N = g.NG;
  cudaStream_t s = H.stream;
  double *S = tmp.get<double>((size_t)n * N);  // first block row, n x 4n
  k_bem_S<<<nblk((int64_t)n * N), 256, 0, s>>>(n, g.h, g.lnh, S);
  FMMPC_LAUNCH_CHECK();
  double *B0 = tmp.get<double>((size_t)n * n), *B2 = tmp.get<double>((size_t)n * n);
  double *E = tmp.get<double>((size_t)4 * n * n);
  k_bem_blocks<<<nblk((int64_t)n * n), 256, 0, s>>>(n, S, B0, B2, E);
  FMMPC_LAUNCH_CHECK();
  const double a0 = gj_invert(B0, n, s, tmp), a2 = gj_invert(B2, n, s, tmp), a1 = gj_invert(E, 2 * n, s, tmp);
  if (!(a0 > 0.0) || !(a2 > 0.0) || !(a1 > 0.0))
    throw Error(FMMPC_ERR_INVALID, "single-layer BEM matrix is singular for this domain");
  H.Sinv = H.pool.get<double>((size_t)n * N);
  k_bem_pack<<<nblk((int64_t)n * n), 256, 0, s>>>(n, B0, B2, E, H.Sinv);
  FMMPC_LAUNCH_CHECK();
  if (H.prec != FMMPC_PREC_FP64) {  // the single-precision forms apply it in two-word FP32
    H.Sinv_hi = H.pool.get<float>((size_t)n * N);
    H.Sinv_lo = H.pool.get<float>((size_t)n * N);
    k_split_f2<<<nblk((int64_t)n * N), 256, 0, s>>>((int64_t)n * N, H.Sinv, H.Sinv_hi, H.Sinv_lo);
    FMMPC_LAUNCH_CHECK();
  }
  FMMPC_CUDA(cudaStreamSynchronize(s));
}

// T' for S^T from T for S (first block rows in the side-DFT form [C0 | C2 | A | B]): S^T is
// block circulant with the blocks transposed and the side index reversed, so its DFT blocks
// are C0^T, C2^T and (A + iB)^H = A^T - i B^T: T'[m][blk n + k] = +-T[k][blk n + m].
__global__ void k_bem_transpose(int n, const double *__restrict__ T, double *__restrict__ Tt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * 4 * n) return;
  const int64_t mrow = t / (4 * n);
  const int c = (int)(t % (4 * n)), blk = c / n, k = c % n;
  const double v = T[(int64_t)k * 4 * n + blk * n + mrow];
  Tt[t] = (blk == 3) ? -v : v;
}

// S^{-T} for the transpose pass, formed on first use.
void init_bem_transpose(fmmpc_handle &H) {
  if (H.SinvT) return;
  const int n = H.g.n;
  double *Tt = H.pool.get<double>((size_t)n * 4 * n);
  k_bem_transpose<<<nblk((int64_t)n * 4 * n), 256, 0, H.stream>>>(n, H.Sinv, Tt);
  FMMPC_LAUNCH_CHECK();
  FMMPC_CUDA(cudaStreamSynchronize(H.stream));
  H.SinvT = Tt;
}

// The inverse of -1/2 I + K in the side-DFT form of the single-layer inverse (the same
// 90-degree rotation symmetry), for the double-layer correction; formed on first use.
void init_bem_dl(fmmpc_handle &H) {
  if (H.Kdl_inv) return;
  const Geo &g = H.g;
  const int n = g.n, N = g.NG;
  cudaStream_t s = H.stream;
  DevPool tmp;
  try {
    double *A = tmp.get<double>((size_t)n * N);
    k_bem_Kdl<<<nblk((int64_t)n * N), 256, 0, s>>>(n, A);
    FMMPC_LAUNCH_CHECK();
    double *B0 = tmp.get<double>((size_t)n * n), *B2 = tmp.get<double>((size_t)n * n);
    double *E = tmp.get<double>((size_t)4 * n * n);
    k_bem_blocks<<<nblk((int64_t)n * n), 256, 0, s>>>(n, A, B0, B2, E);
    FMMPC_LAUNCH_CHECK();
    const double a0 = gj_invert(B0, n, s, tmp), a2 = gj_invert(B2, n, s, tmp), a1 = gj_invert(E, 2 * n, s, tmp);
    if (!(a0 > 0.0) || !(a2 > 0.0) || !(a1 > 0.0))
      throw Error(FMMPC_ERR_INVALID, "double-layer BEM matrix is singular for this domain");
    double *T = H.pool.get<double>((size_t)n * N);
    k_bem_pack<<<nblk((int64_t)n * n), 256, 0, s>>>(n, B0, B2, E, T);
    FMMPC_LAUNCH_CHECK();
    float *th = nullptr, *tl = nullptr;
    if (H.prec != FMMPC_PREC_FP64) {
      th = H.pool.get<float>((size_t)n * N);
      tl = H.pool.get<float>((size_t)n * N);
      k_split_f2<<<nblk((int64_t)n * N), 256, 0, s>>>((int64_t)n * N, T, th, tl);
      FMMPC_LAUNCH_CHECK();
    }
    FMMPC_CUDA(cudaStreamSynchronize(s));
    H.Kdl_inv = T;
    H.Kdl_hi = th;
    H.Kdl_lo = tl;
  } catch (...) {
    cudaStreamSynchronize(s);
    throw;
  }
}

}  // namespace fmmpc
