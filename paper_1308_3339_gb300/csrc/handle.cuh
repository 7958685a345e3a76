// The handle behind the C ABI: geometry, tree, lists, FMM and BEM buffers, Krylov
// workspace.  Shared by api.cu, fmm.cu and krylov.cu.
#pragma once

#include <string>

#include "common.cuh"

namespace fmmpc {

enum ApplyPart {
  PART_FULL = 0,   // P^{-1} r
  PART_VR = 1,     // V r at the nodes
  PART_NEAR = 2,   // near-field (P2P) part of V r, physical units
  PART_VCOL = 3,   // V r at the collocation points
  PART_Q = 4,      // BEM density q (mu in the double-layer form)
  PART_BC = 5,     // the boundary-integral solution with Dirichlet data H.bc_g (fmmpc_apply_bc)
  PART_TRANS = 6,  // the transpose P^{-T} (fmmpc_apply_transpose)
};

// FMM buffers for one arithmetic type (float or double).
struct FmmBufs {
  void *wpad = nullptr;      // [nrhs][npad^2] padded weight image h^2 r
  void *Mv = nullptr;        // [nrhs][ncell][p] volume multipoles
  void *Lv = nullptr;        // [nrhs][ncell][p] volume locals
  void *Mb = nullptr;        // [nrhs][nbcell][p] boundary multipoles
  void *Lb = nullptr;        // [nrhs][nbcell][p] boundary locals
  void *phib = nullptr;      // [nrhs][nbnear][m^2] near-boundary correction at nodes
  void *table = nullptr;     // lattice table ln|d| (node units), self term at d = 0
  void *mats = nullptr;      // fixed M2M / L2L / boundary P2M translation matrices
  void *table_lnh = nullptr; // same plus ln h (for the near-field-only part)
  int table_rows = 0, table_stride = 0, table_c0 = 0, Rn = 0;
  double *vcol = nullptr;    // [nrhs][NG] V r at collocation points
  double *q = nullptr;       // [nrhs][NG] BEM density
  double *vt = nullptr;      // [nrhs][NG] side-DFT of vcol for the block-circulant apply
  float *vt_hi = nullptr, *vt_lo = nullptr;  // the same as two FP32 words (single-precision forms)
  float *knear = nullptr;    // near-boundary element integrals (single-precision forms)
  float *kcol = nullptr;     // collocation-point near-field log kernel (single-precision forms)
  void *vnear = nullptr;     // [nrhs][NG] near part of V r at the collocation points (R)
  void *Lvb = nullptr;       // [nrhs][n_vbv_cells][p] boundary-source part of L of those cells
  int *up_count = nullptr;   // [nrhs][up_ncount] upward-pass arrival counts (zero between launches)
  int64_t up_ncount = 0;
  int bup_lc = 0;            // boundary upward pass: levels whose cells are split into chunks
  void *bup_part = nullptr;  // [nrhs][bup_lc n/64][p] chunk partial multipoles
  int *bup_cnt = nullptr;    // [nrhs][coarse boundary cells] arrival counts (zero between launches)
};

// tensor-core lattice P2P (p2p_tc.cu)
struct TcP2P {
  bool enabled = false;
  int NLX = 0, NLY = 0, NS = 0, npass = 3, nrows = 0, nofs = 0, smem = 0, usplit = 0;
  int row_oy[33] = {}, row_q0[33] = {}, row_q1[33] = {}, row_ox0[33] = {};
  uint16_t *ahi = nullptr, *alo = nullptr;        // FP16 weight strips (scaled), hi and lo words
  uint16_t *bmat = nullptr, *bmat_lnh = nullptr;  // FP16 kernel tables, hi and lo words
  float *near1 = nullptr, *near2 = nullptr;  // the two halves of the near-field sum, FP32 images
  float *lsc = nullptr;                      // [nrhs][NLY][NLX] 2^-e of each leaf's FP16 weights
  int *err = nullptr;
};

// tensor-core M2L for the mixed-precision forms (m2l_tc.cu)
struct TcM2L {
  bool enabled = false;
  int kind = 0;  // 0 TF32, 1 BF16
  int nsplit = 0;  // leading multipoles split hi + lo
  int sbase = 0;   // first K column of the split products
  int width = 32;  // outputs per target class (N = 4 width)
  int ntiles = 0, smem = 0, nofs_total = 0;  // nofs_total: shifts
  int nparts = 1, gpart[3] = {}, gpart_sh[3] = {};
  int64_t rows_per_rhs = 0;
  int64_t lev_row0[24] = {};
  int lev_P[24] = {};
  unsigned char *img = nullptr, *bmat = nullptr;
  int2 *tiles = nullptr;
  int4 *groups = nullptr;
  int *dxs = nullptr, *err = nullptr;
};

struct GraphEntry {
  const double *r;
  double *out;
  int nrhs;
  int timing;
  cudaGraphExec_t exec;
  uint64_t last;
};

struct KrylovWs {
  int64_t cap_vecs = 0;   // vectors of N*nrhs doubles allocated in V (and Z)
  double *V = nullptr, *Z = nullptr;
  double *w = nullptr, *t = nullptr, *b = nullptr, *x = nullptr, *r = nullptr;
  double *fin = nullptr, *gin = nullptr, *zin = nullptr;  // graph solves: f, g, z_j
  double *dots = nullptr;  // [4][nrhs][MAXDOT]
  double *part = nullptr;  // block partials
  double *scal = nullptr;  // per-rhs scalars on device
  double *hbuf = nullptr;  // pinned host mirror
  int *mask = nullptr;     // [nrhs] active right-hand sides
  // device-resident state of the graph solves (krylov.cu)
  int *g_ctl = nullptr, *g_done = nullptr, *g_iters = nullptr;
  int *g_cnt = nullptr;  // [nrhs] arrival counters of the fused reductions (zero between launches)
  double *g_H = nullptr, *g_cs = nullptr, *g_sn = nullptr, *g_g = nullptr, *g_bn = nullptr, *g_rel = nullptr,
         *g_sc = nullptr, *g_rtol = nullptr;
};

// An instantiated whole-solve graph (krylov.cu), keyed by method, restart, right-hand
// sides, boundary data present, and the number of problems it solves side by side.
struct SolveGraph {
  int method, m, nrhs, has_g, nprob;
  cudaGraphExec_t exec;
  std::vector<uint64_t> gens;  // workspace generation of every member handle when built
};

}  // namespace fmmpc

struct fmmpc_handle {
  fmmpc::Geo g{};
  fmmpc::Stencil st{};
  int prec = FMMPC_PREC_FP32;
  int nrhs_max = 1;
  int tile_x = 8, tile_y = 4;
  cudaStream_t stream = nullptr;
  std::string err;
  fmmpc::DevPool pool;      // lifetime of the handle
  fmmpc::DevPool kpool;     // Krylov workspace (grown on demand)
  fmmpc::TreeOut tree{};
  fmmpc::Lists lists{};
  fmmpc::FmmBufs fb{};
  double *Sinv = nullptr;   // [n][4n] first block row of the FP64 inverse of the single-layer matrix
  double *Kdl_inv = nullptr;  // the same for -1/2 I + K (double-layer correction), made on first use
  double *SinvT = nullptr;    // the same for S^T (the transpose pass), made on first use
  float *Kdl_hi = nullptr, *Kdl_lo = nullptr;  // and as two FP32 words (single-precision forms)
  int bem_form = 0;         // 0: single-layer correction (Eq. e:ubound), 1: second-kind double layer
  const double *bc_g = nullptr;  // boundary data of the running fmmpc_apply_bc call (else NULL)
  bool trans_pass = false;       // the running apply is the transpose pass
  float *Sinv_hi = nullptr, *Sinv_lo = nullptr;  // the same as two FP32 words (single-precision forms)
  double *stage_in = nullptr, *stage_out = nullptr, *stage_g = nullptr;  // device staging for *_host calls
  fmmpc::KrylovWs kw{};
  fmmpc::TcP2P tcp{};
  fmmpc::TcM2L tcm{};
  int p2p_engine = 0;       // 0: tensor cores where eligible, 1: CUDA cores
  // operator of the Krylov solves (fmmpc_set_operator): 0 five-point, 1 five-point with the
  // coefficient acoef [(n+2)^2], 2 Q1 stiffness (q1tab: Thomas coefficients of the mass solve)
  int op = 0;
  double *acoef = nullptr, *q1tab = nullptr;
  int64_t launches = 0;     // kernel launches of the last apply
  // optional per-stage CUDA-event timing of the apply (fmmpc_set_timing)
  static constexpr int NSTAGE = 11;
  int timing = 0;  // 0 off, 1 every stage, 2 only the M2L and P2P kernels (four events)
  cudaEvent_t ev[NSTAGE + 1] = {};
  bool stage_hit[NSTAGE] = {};
  double t_setup_ms = 0.0;
  // CUDA graphs of the full apply, replayed on an internal stream (fmmpc_set_graphs)
  bool graphs = true;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  cudaStream_t sstream = nullptr;   // second stream of the full apply (near field, volume M2L)
  cudaStream_t sstream2 = nullptr;  // third stream (near-boundary correction)
  cudaStream_t sstream3 = nullptr;  // fourth stream (volume M2L)
  cudaEvent_t sev[7] = {};  // forks after the weights, the upward pass and the BEM solve; four joins
  std::vector<fmmpc::GraphEntry> gcache;
  uint64_t gclock = 0;
  // whole-solve graphs (device-resident Krylov loop) and the stream they are captured on
  std::vector<fmmpc::SolveGraph> sgraphs;
  cudaStream_t cstream = nullptr;
  uint64_t ws_gen = 0;  // bumped whenever the Krylov workspace is reallocated
};

namespace fmmpc {
void apply_fmm(fmmpc_handle &H, int part, const double *r, double *out, int nrhs);
// the apply's kernels issued on H.stream one by one (no graph of its own; used inside captures)
void apply_fmm_eager(fmmpc_handle &H, int part, const double *r, double *out, int nrhs);
void clear_solve_graphs(fmmpc_handle &H);
void precond_op(fmmpc_handle &H, const double *r, double *z, double *scratch, int nrhs, bool in_capture);
void q1_mass_solve(fmmpc_handle &H, const double *r, double *c, int nrhs);
int solve_graphed(fmmpc_handle &H, const double *f, const double *g, double *u, int nrhs, const fmmpc_solve_opts &o,
                  fmmpc_solve_info &info);
cudaGraphExec_t solve_graph(std::vector<fmmpc_handle *> &hs, int method, int m, int nrhs, bool has_g);
int solve_batched_graphed(std::vector<fmmpc_handle *> &hs, const double *const *f, const double *const *gb,
                          double *const *u, const fmmpc_solve_opts &o, fmmpc_solve_info *infos);
void init_fmm(fmmpc_handle &H);
void init_bem(fmmpc_handle &H, DevPool &tmp);
void init_bem_dl(fmmpc_handle &H);
void init_bem_transpose(fmmpc_handle &H);
void spmv5(fmmpc_handle &H, const double *x, double *y, int nrhs);
int solve(fmmpc_handle &H, const double *f, const double *g, double *u, int nrhs,
          const fmmpc_solve_opts &o, fmmpc_solve_info &info);
bool tc_p2p_eligible(const fmmpc_handle &H);
void init_tc_p2p(fmmpc_handle &H);
int prep_p2p_tc(fmmpc_handle &H, const double *r, int nrhs, cudaStream_t s, float *wimg);
bool tc_m2l_eligible(const fmmpc_handle &H);
void init_tc_m2l(fmmpc_handle &H, DevPool &tmp);
int run_m2l_tc(fmmpc_handle &H, const void *Mv, void *Lv, int nrhs, cudaStream_t s);
int run_p2p_tc(fmmpc_handle &H, bool with_lnh, double *out, int nrhs, cudaStream_t s);
int add_near2(fmmpc_handle &H, double *out, int nrhs, cudaStream_t s);
// message for fmmpc_last_error(NULL), kept in a fixed thread-local buffer; returns code
int set_global_error(int code, const char *msg);
int solve_batched(std::vector<fmmpc_handle *> &hs, const double *const *f, const double *const *gb,
                  double *const *u, const fmmpc_solve_opts &o, fmmpc_solve_info *infos);
int autotune(const fmmpc_grid &g, const fmmpc_params &base, const fmmpc_solve_opts &opts, const double *f_dev,
             double tol, void *stream, fmmpc_params &best, std::vector<fmmpc_tune_entry> &report, bool want_report);
int create_handle(fmmpc_handle **out, const fmmpc_grid &g, const fmmpc_params &p, void *stream);
int near_field_noalloc(int32_t n, double side, int32_t leaf_max, double theta, const double *r_dev,
                       double *out_dev, void *stream);
}  // namespace fmmpc
