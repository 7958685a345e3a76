// Boundary-element set-up (Sec. 4.3): constant elements, no nodes at the corners, 4n
// equal elements on the square, collocation at their midpoints.  The single-layer
// matrix S_mk = int_{Gamma_k} G(y_m, y) dGamma (left side of Eq. e:ubound) is assembled in
// FP64 from the closed-form element integral (Sec. 4.2).  The square's 90-degree rotation
// symmetry makes S block circulant over the four sides, so a 4-point DFT over the side
// index splits it into three n x n blocks (one complex); each is inverted once (LU with
// partial pivoting by cuSOLVER, then the triangular solves against the identity), and the
// apply works in that basis.  The inversion is set-up, not the apply's path.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
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

// From the first block row of S (n x 4n): S^0 and S^2 (n x n, real) and
// S^1 = (S0 - S2) + i (S1 - S3) (n x n, complex, interleaved re / im).
__global__ void k_bem_blocks(int n, const double *__restrict__ S, double *__restrict__ B0, double *__restrict__ B2,
                             double *__restrict__ C1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int64_t m = t / n;
  const int k = (int)(t % n);
  const double *row = S + m * 4 * n;
  const double s0 = row[k], s1 = row[n + k], s2 = row[2 * n + k], s3 = row[3 * n + k];
  B0[m * n + k] = (s0 + s2) + (s1 + s3);
  B2[m * n + k] = (s0 + s2) - (s1 + s3);
  C1[2 * (m * n + k)] = s0 - s2;
  C1[2 * (m * n + k) + 1] = s1 - s3;
}

// T[m] = [inv(S^0) | inv(S^2) | A | B][m] with A + i B = inv(S^1).
__global__ void k_bem_pack(int n, const double *__restrict__ B0, const double *__restrict__ B2,
                           const double *__restrict__ C1, double *__restrict__ T) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int64_t m = t / n;
  const int k = (int)(t % n);
  double *o = T + m * 4 * n;
  o[k] = B0[m * n + k];
  o[n + k] = B2[m * n + k];
  o[2 * n + k] = C1[2 * (m * n + k)];
  o[3 * n + k] = C1[2 * (m * n + k) + 1];
}

__global__ void k_identity(int N, double *__restrict__ B, int cplx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const double v = (t / N == t % N) ? 1.0 : 0.0;
  if (cplx) {
    B[2 * t] = v;
    B[2 * t + 1] = 0.0;
  } else {
    B[t] = v;
  }
}

// |A_kk| of the N x N (real or interleaved complex) matrix A
__global__ void k_diag_abs(int N, const double *__restrict__ A, double *__restrict__ d, int cplx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t i = (int64_t)k * N + k;
  d[k] = cplx ? hypot(A[2 * i], A[2 * i + 1]) : fabs(A[i]);
}

#define FMMPC_CUSOLVER(call)                                                                   \
  do {                                                                                          \
    const cusolverStatus_t st_ = (call);                                                        \
    if (st_ != CUSOLVER_STATUS_SUCCESS)                                                         \
      throw ::fmmpc::Error(FMMPC_ERR_CUDA, std::string(#call) + ": cuSOLVER status " + std::to_string((int)st_)); \
  } while (0)

// One cuSOLVER handle per device for the process (creating one costs milliseconds).
cusolverDnHandle_t solver_handle() {
  static std::mutex mu;
  static std::map<int, cusolverDnHandle_t> handles;
  int dev = 0;
  FMMPC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = handles.find(dev);
  if (it != handles.end()) return it->second;
  cusolverDnHandle_t h = nullptr;
  FMMPC_CUSOLVER(cusolverDnCreate(&h));
  handles[dev] = h;
  return h;
}

// In-place inverse of the N x N matrix A (row-major, device; real, or complex with re / im
// interleaved), by LU with partial pivoting and the two triangular solves against the
// identity.  Row-major A is the column-major A^T, and inv(A^T) read row-major is inv(A), so
// the factorisation runs on the buffer as it is.  Returns the smallest |U_kk| (0 for a
// singular matrix).  Calls are serialised on the handle's stream.
double lu_invert(double *A, int N, bool cplx, cudaStream_t s, DevPool &tmp) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);  // the per-device solver handle is shared
  cusolverDnHandle_t h = solver_handle();
  FMMPC_CUSOLVER(cusolverDnSetStream(h, s));
  const size_t w = cplx ? 2 : 1;
  int lwork = 0;
  cuDoubleComplex *Az = reinterpret_cast<cuDoubleComplex *>(A);
  if (cplx) FMMPC_CUSOLVER(cusolverDnZgetrf_bufferSize(h, N, N, Az, N, &lwork));
  else FMMPC_CUSOLVER(cusolverDnDgetrf_bufferSize(h, N, N, A, N, &lwork));
  double *work = tmp.get<double>(w * (size_t)std::max(lwork, 1));
  int *ipiv = tmp.get<int>(N), *info = tmp.get<int>(2);
  double *dabs = tmp.get<double>(N), *B = tmp.get<double>(w * (size_t)N * N);
  if (cplx) FMMPC_CUSOLVER(cusolverDnZgetrf(h, N, N, Az, N, reinterpret_cast<cuDoubleComplex *>(work), ipiv, info));
  else FMMPC_CUSOLVER(cusolverDnDgetrf(h, N, N, A, N, work, ipiv, info));
  k_diag_abs<<<nblk(N), 256, 0, s>>>(N, A, dabs, cplx ? 1 : 0);
  k_identity<<<nblk((int64_t)N * N), 256, 0, s>>>(N, B, cplx ? 1 : 0);
  FMMPC_LAUNCH_CHECK();
  if (cplx)
    FMMPC_CUSOLVER(cusolverDnZgetrs(h, CUBLAS_OP_N, N, N, Az, N, ipiv, reinterpret_cast<cuDoubleComplex *>(B), N,
                                    info + 1));
  else
    FMMPC_CUSOLVER(cusolverDnDgetrs(h, CUBLAS_OP_N, N, N, A, N, ipiv, B, N, info + 1));
  FMMPC_CUDA(cudaMemcpyAsync(A, B, sizeof(double) * w * N * N, cudaMemcpyDeviceToDevice, s));
  std::vector<double> ha(N);
  int hinfo[2] = {0, 0};
  FMMPC_CUDA(cudaMemcpyAsync(ha.data(), dabs, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaMemcpyAsync(hinfo, info, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaStreamSynchronize(s));
  if (hinfo[0] > 0) return 0.0;  // U_kk == 0 at k = info - 1
  if (hinfo[0] < 0 || hinfo[1] != 0)
    throw Error(FMMPC_ERR_CUDA, "cuSOLVER getrf/getrs: invalid argument " + std::to_string(hinfo[0] ? hinfo[0] : hinfo[1]));
  double amin = ha[0];
  for (int k = 0; k < N; ++k) amin = std::min(amin, ha[k]);
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
  // of S is assembled and three n x n systems are inverted (two real, one complex).
  const Geo &g = H.g;
  const int n = g.n, N = g.NG;
  cudaStream_t s = H.stream;
  double *S = tmp.get<double>((size_t)n * N);  // first block row, n x 4n
  k_bem_S<<<nblk((int64_t)n * N), 256, 0, s>>>(n, g.h, g.lnh, S);
  FMMPC_LAUNCH_CHECK();
  double *B0 = tmp.get<double>((size_t)n * n), *B2 = tmp.get<double>((size_t)n * n);
  double *C1 = tmp.get<double>((size_t)2 * n * n);
  k_bem_blocks<<<nblk((int64_t)n * n), 256, 0, s>>>(n, S, B0, B2, C1);
  FMMPC_LAUNCH_CHECK();
  const double a0 = lu_invert(B0, n, false, s, tmp), a2 = lu_invert(B2, n, false, s, tmp), a1 = lu_invert(C1, n, true, s, tmp);
  if (!(a0 > 0.0) || !(a2 > 0.0) || !(a1 > 0.0))
    throw Error(FMMPC_ERR_INVALID, "single-layer BEM matrix is singular for this domain");
  H.Sinv = H.pool.get<double>((size_t)n * N);
  k_bem_pack<<<nblk((int64_t)n * n), 256, 0, s>>>(n, B0, B2, C1, H.Sinv);
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
    double *C1 = tmp.get<double>((size_t)2 * n * n);
    k_bem_blocks<<<nblk((int64_t)n * n), 256, 0, s>>>(n, A, B0, B2, C1);
    FMMPC_LAUNCH_CHECK();
    const double a0 = lu_invert(B0, n, false, s, tmp), a2 = lu_invert(B2, n, false, s, tmp), a1 = lu_invert(C1, n, true, s, tmp);
    if (!(a0 > 0.0) || !(a2 > 0.0) || !(a1 > 0.0))
      throw Error(FMMPC_ERR_INVALID, "double-layer BEM matrix is singular for this domain");
    double *T = H.pool.get<double>((size_t)n * N);
    k_bem_pack<<<nblk((int64_t)n * n), 256, 0, s>>>(n, B0, B2, C1, T);
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
