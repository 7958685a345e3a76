// Quadtree and interaction lists on the GPU.
//
// Tree (Sec. 5.1): Morton keys of the nodes, a stable radix sort into Morton order, and
// the start of every cell at every level, read off where the key prefix changes.
// Lists (Sec. 5.2): the dual tree traversal from (root, root), run level by level as a
// frontier of cell pairs.  A pair that meets the multipole acceptance criterion
// (R_A + R_B) < theta |c_A - c_B| becomes an M2L pair, a pair of leaves that does not
// becomes a P2P pair, anything else is replaced by all pairs of children.  The MAC is
// evaluated exactly in integers (theta = tnum/tden, lengths in h/2 or h/2^(L+1) units)
// so rounding never decides membership.  A second traversal pairs volume cells with
// boundary cells (runs of elements along one side, bounded by their circumscribed
// square).  The lists are then radix-sorted into (level, target, source) order.
#include <algorithm>
#include <map>
#include <set>

#include "common.cuh"

namespace fmmpc {

namespace {

__global__ void k_morton_keys(int n, uint32_t *__restrict__ keys, uint64_t *__restrict__ k64,
                              uint32_t *__restrict__ idx) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t % n), j = (int)(t / n);
  uint32_t k = morton_encode((uint32_t)i, (uint32_t)j);
  keys[t] = k;
  k64[t] = k;
  idx[t] = (uint32_t)t;
}

__global__ void k_cell_starts(const uint64_t *__restrict__ sk, int64_t N, int L, int lg,
                              int32_t *__restrict__ start) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  for (int l = 0; l <= L; ++l) {
    int sh = 2 * (lg - l);
    uint64_t c = sk[k] >> sh;
    if (k == 0 || (sk[k - 1] >> sh) != c) start[level_offset(l) + (int64_t)c] = (int32_t)k;
  }
}

__device__ __forceinline__ bool mac_int(const GeoDev &g, int64_t dx, int64_t dy, int64_t ssum) {
  __int128 d2 = (__int128)dx * dx + (__int128)dy * dy;
  __int128 lhs = (__int128)2 * g.tden * g.tden * (__int128)ssum * ssum;
  return lhs < (__int128)g.tnum * g.tnum * d2;
}

// kind 0: volume-volume pairs (A, B), 16 children; kind 1: volume-boundary (v, b), 8 children
template <int KIND>
__global__ void k_dtt_classify(GeoDev g, int l, const uint32_t *__restrict__ fa,
                               const uint32_t *__restrict__ fb, int64_t nf, int32_t *__restrict__ cm2l,
                               int32_t *__restrict__ cp2p, int32_t *__restrict__ cch) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  int64_t XA, YA, sA, XB, YB, sB;
  vol_geom(g, l, fa[t], XA, YA, sA);
  bool mac;
  if (KIND == 0) {
    vol_geom(g, l, fb[t], XB, YB, sB);
    mac = mac_int(g, XA - XB, YA - YB, sA + sB);
  } else {
    bnd_geom(g, l, fb[t], XB, YB, sB);
    XA <<= g.L; YA <<= g.L; sA <<= g.L;
    mac = mac_int(g, XA - XB, YA - YB, sA + sB);
  }
  int m = 0, p = 0, c = 0;
  if (mac) m = 1;
  else if (l == g.L) p = 1;
  else c = (KIND == 0) ? 16 : 8;
  cm2l[t] = m;
  cp2p[t] = p;
  cch[t] = c;
}

template <int KIND>
__global__ void k_dtt_emit(int l, const uint32_t *__restrict__ fa, const uint32_t *__restrict__ fb,
                           int64_t nf, const int32_t *__restrict__ cm2l, const int32_t *__restrict__ om2l,
                           const int32_t *__restrict__ cp2p, const int32_t *__restrict__ op2p,
                           const int32_t *__restrict__ cch, const int32_t *__restrict__ och,
                           uint64_t *__restrict__ m2l_out, uint64_t *__restrict__ p2p_out,
                           uint32_t *__restrict__ na, uint32_t *__restrict__ nb) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  uint32_t A = fa[t], B = fb[t];
  // keys: level(5) | target(27) | source(27) for M2L, target | source for P2P
  if (cm2l[t]) m2l_out[om2l[t]] = ((uint64_t)l << 54) | ((uint64_t)A << 27) | B;
  if (cp2p[t]) p2p_out[op2p[t]] = ((uint64_t)A << 27) | B;
  if (cch[t]) {
    int64_t o = och[t];
    if (KIND == 0) {
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          na[o] = 4 * A + i;
          nb[o] = 4 * B + j;
          ++o;
        }
    } else {
      uint32_t side = B >> l, k = B & ((1u << l) - 1u);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 2; ++j) {
          na[o] = 4 * A + i;
          nb[o] = (side << (l + 1)) + 2 * k + j;
          ++o;
        }
    }
  }
}

__global__ void k_decode3(const uint64_t *__restrict__ key, int64_t n, int32_t *__restrict__ out,
                          int swap_ts) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t k = key[e];
  int32_t l = (int32_t)(k >> 54), a = (int32_t)((k >> 27) & 0x7ffffff), b = (int32_t)(k & 0x7ffffff);
  out[3 * e] = l;
  out[3 * e + 1] = swap_ts ? b : a;
  out[3 * e + 2] = swap_ts ? a : b;
}
__global__ void k_decode2(const uint64_t *__restrict__ key, int64_t n, int32_t *__restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t k = key[e];
  out[2 * e] = (int32_t)((k >> 27) & 0x7ffffff);
  out[2 * e + 1] = (int32_t)(k & 0x7ffffff);
}
// swap (target, source) of M2L/P2P keys so the list can be regrouped by source
__global__ void k_swap_key3(const uint64_t *__restrict__ in, int64_t n, uint64_t *__restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t k = in[e];
  uint64_t l = k >> 54, a = (k >> 27) & 0x7ffffff, b = k & 0x7ffffff;
  out[e] = (l << 54) | (b << 27) | a;
}

// CSR counts: count[group(e)] += 1 where group = level_offset(level) + target
__global__ void k_group_count(const int32_t *__restrict__ ent, int64_t n, int width, int tcol,
                              int lcol, int boundary, int32_t *__restrict__ count,
                              int32_t *__restrict__ src, int scol) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t *r = ent + width * e;
  int64_t g = r[tcol];
  if (lcol >= 0) g += boundary ? blevel_offset(r[lcol]) : level_offset(r[lcol]);
  atomicAdd(&count[g], 1);
  src[e] = r[scol];
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct LevelOut {
  uint64_t *m2l;
  int64_t nm2l;
  uint64_t *p2p;
  int64_t np2p;
};

// Level-synchronous dual tree traversal. Returns unsorted keys of all M2L and P2P pairs.
template <int KIND>
void traverse(const Geo &geo, cudaStream_t s, DevPool &tmp, uint64_t *&m2l_keys, int64_t &nm2l,
              uint64_t *&p2p_keys, int64_t &np2p, const std::vector<uint32_t> &root_a,
              const std::vector<uint32_t> &root_b) {
  GeoDev g{geo.n, geo.L, geo.tnum, geo.tden};
  int64_t nf = (int64_t)root_a.size();
  uint32_t *fa = tmp.get<uint32_t>(nf), *fb = tmp.get<uint32_t>(nf);
  FMMPC_CUDA(cudaMemcpyAsync(fa, root_a.data(), 4 * nf, cudaMemcpyHostToDevice, s));
  FMMPC_CUDA(cudaMemcpyAsync(fb, root_b.data(), 4 * nf, cudaMemcpyHostToDevice, s));
  std::vector<LevelOut> outs;
  for (int l = 0; l <= geo.L && nf > 0; ++l) {
    int32_t *cm = tmp.get<int32_t>(nf), *cp = tmp.get<int32_t>(nf), *cc = tmp.get<int32_t>(nf);
    int32_t *om = tmp.get<int32_t>(nf), *op = tmp.get<int32_t>(nf), *oc = tmp.get<int32_t>(nf);
    k_dtt_classify<KIND><<<blocks(nf), 256, 0, s>>>(g, l, fa, fb, nf, cm, cp, cc);
    FMMPC_LAUNCH_CHECK();
    int32_t tm = 0, tp = 0, tc = 0;
    scan_exclusive_i32(cm, om, nf, &tm, s, tmp);
    scan_exclusive_i32(cp, op, nf, &tp, s, tmp);
    scan_exclusive_i32(cc, oc, nf, &tc, s, tmp);
    LevelOut lo{tmp.get<uint64_t>(tm + 1), tm, tmp.get<uint64_t>(tp + 1), tp};
    uint32_t *na = tmp.get<uint32_t>(tc + 1), *nb = tmp.get<uint32_t>(tc + 1);
    k_dtt_emit<KIND><<<blocks(nf), 256, 0, s>>>(l, fa, fb, nf, cm, om, cp, op, cc, oc, lo.m2l, lo.p2p, na, nb);
    FMMPC_LAUNCH_CHECK();
    outs.push_back(lo);
    fa = na;
    fb = nb;
    nf = tc;
  }
  nm2l = 0;
  np2p = 0;
  for (auto &o : outs) { nm2l += o.nm2l; np2p += o.np2p; }
  m2l_keys = tmp.get<uint64_t>(nm2l + 1);
  p2p_keys = tmp.get<uint64_t>(np2p + 1);
  int64_t a = 0, b = 0;
  for (auto &o : outs) {
    if (o.nm2l) FMMPC_CUDA(cudaMemcpyAsync(m2l_keys + a, o.m2l, 8 * o.nm2l, cudaMemcpyDeviceToDevice, s));
    if (o.np2p) FMMPC_CUDA(cudaMemcpyAsync(p2p_keys + b, o.p2p, 8 * o.np2p, cudaMemcpyDeviceToDevice, s));
    a += o.nm2l;
    b += o.np2p;
  }
}

void sort_keys(uint64_t *keys, int64_t n, int bits, cudaStream_t s, DevPool &tmp) {
  if (n <= 1) return;
  uint32_t *dummy = tmp.get<uint32_t>(n);
  radix_sort_u64(keys, dummy, n, bits, s, tmp);
}

// CSR over groups: first[g] for g in [0, ngroups], src[e] = column scol of entry e.
void build_csr(const int32_t *ent, int64_t n, int width, int tcol, int lcol, int boundary, int scol,
               int64_t ngroups, int32_t *first, int32_t *src, cudaStream_t s, DevPool &tmp) {
  int32_t *count = tmp.get<int32_t>(ngroups + 1);
  FMMPC_CUDA(cudaMemsetAsync(count, 0, 4 * (ngroups + 1), s));
  if (n > 0) {
    k_group_count<<<blocks(n), 256, 0, s>>>(ent, n, width, tcol, lcol, boundary, count, src, scol);
    FMMPC_LAUNCH_CHECK();
  }
  scan_exclusive_i32(count, first, ngroups + 1, nullptr, s, tmp);
}

}  // namespace

void build_tree(const Geo &g, TreeOut &t, cudaStream_t s, DevPool &pool, DevPool &tmp) {
  const int64_t N = (int64_t)g.n * g.n;
  t.keys = pool.get<uint32_t>(N);
  t.perm = pool.get<int32_t>(N);
  t.cell_start = pool.get<int32_t>(g.ncell);
  uint64_t *k64 = tmp.get<uint64_t>(N);
  uint32_t *idx = tmp.get<uint32_t>(N);
  k_morton_keys<<<blocks(N), 256, 0, s>>>(g.n, t.keys, k64, idx);
  FMMPC_LAUNCH_CHECK();
  radix_sort_u64(k64, idx, N, 2 * g.lg, s, tmp);
  FMMPC_CUDA(cudaMemcpyAsync(t.perm, idx, 4 * N, cudaMemcpyDeviceToDevice, s));
  FMMPC_CUDA(cudaMemsetAsync(t.cell_start, 0xff, 4 * g.ncell, s));
  k_cell_starts<<<blocks(N), 256, 0, s>>>(k64, N, g.L, g.lg, t.cell_start);
  FMMPC_LAUNCH_CHECK();
  // the kernels below assume the complete tree of an m 2^L grid: check it
  std::vector<int32_t> st(g.ncell);
  FMMPC_CUDA(cudaMemcpyAsync(st.data(), t.cell_start, 4 * g.ncell, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l <= g.L; ++l) {
    int64_t w = g.n >> l, nc = int64_t(1) << (2 * l);
    for (int64_t c = 0; c < nc; ++c)
      if (st[level_offset(l) + c] != (int32_t)(c * w * w))
        throw Error(FMMPC_ERR_INVALID, "tree: cell ranges are not those of a complete quadtree");
  }
}

void build_lists(const Geo &g, Lists &Ls, Stencil &st, cudaStream_t s, DevPool &pool, DevPool &tmp) {
  // ---- volume-volume traversal
  uint64_t *m2l_k, *p2p_k;
  int64_t nm2l, np2p;
  traverse<0>(g, s, tmp, m2l_k, nm2l, p2p_k, np2p, {0u}, {0u});
  sort_keys(m2l_k, nm2l, 58, s, tmp);
  sort_keys(p2p_k, np2p, 54, s, tmp);
  Ls.n_m2l = nm2l;
  Ls.n_p2p = np2p;
  Ls.m2l = pool.get<int32_t>(3 * nm2l + 3);
  Ls.p2p = pool.get<int32_t>(2 * np2p + 2);
  if (nm2l) k_decode3<<<blocks(nm2l), 256, 0, s>>>(m2l_k, nm2l, Ls.m2l, 0);
  if (np2p) k_decode2<<<blocks(np2p), 256, 0, s>>>(p2p_k, np2p, Ls.p2p);
  FMMPC_LAUNCH_CHECK();
  // ---- volume-boundary traversal: (volume root, root run of each side)
  uint64_t *vb_k, *pvb_k;
  int64_t nvb, npvb;
  traverse<1>(g, s, tmp, vb_k, nvb, pvb_k, npvb, {0u, 0u, 0u, 0u}, {0u, 1u, 2u, 3u});
  sort_keys(vb_k, nvb, 58, s, tmp);
  sort_keys(pvb_k, npvb, 54, s, tmp);
  Ls.n_m2l_vb = nvb;
  Ls.n_p2p_vb = npvb;
  Ls.m2l_vb = pool.get<int32_t>(3 * nvb + 3);
  Ls.p2p_vb = pool.get<int32_t>(2 * npvb + 2);
  if (nvb) k_decode3<<<blocks(nvb), 256, 0, s>>>(vb_k, nvb, Ls.m2l_vb, 0);
  if (npvb) k_decode2<<<blocks(npvb), 256, 0, s>>>(pvb_k, npvb, Ls.p2p_vb);
  FMMPC_LAUNCH_CHECK();

  // ---- CSR views
  Ls.m2l_first = pool.get<int32_t>(g.ncell + 1);
  Ls.m2l_src = pool.get<int32_t>(nm2l + 1);
  build_csr(Ls.m2l, nm2l, 3, 1, 0, 0, 2, g.ncell, Ls.m2l_first, Ls.m2l_src, s, tmp);
  Ls.vbv_first = pool.get<int32_t>(g.ncell + 1);
  Ls.vbv_src = pool.get<int32_t>(nvb + 1);
  build_csr(Ls.m2l_vb, nvb, 3, 1, 0, 0, 2, g.ncell, Ls.vbv_first, Ls.vbv_src, s, tmp);
  {
    // the volume cells that have boundary M2L sources, for passes that only add those
    std::vector<int32_t> hf(g.ncell + 1), cells;
    FMMPC_CUDA(cudaMemcpyAsync(hf.data(), Ls.vbv_first, sizeof(int32_t) * (g.ncell + 1), cudaMemcpyDeviceToHost, s));
    FMMPC_CUDA(cudaStreamSynchronize(s));
    for (int64_t c = 0; c < g.ncell; ++c)
      if (hf[c + 1] > hf[c]) cells.push_back((int32_t)c);
    Ls.n_vbv_cells = (int64_t)cells.size();
    Ls.vbv_cells = pool.get<int32_t>(cells.size() + 1);
    if (!cells.empty())
      FMMPC_CUDA(cudaMemcpyAsync(Ls.vbv_cells, cells.data(), sizeof(int32_t) * cells.size(), cudaMemcpyHostToDevice, s));
    std::vector<int32_t> slot(g.ncell, -1);  // cell -> its index in vbv_cells
    for (size_t i = 0; i < cells.size(); ++i) slot[cells[i]] = (int32_t)i;
    Ls.vbv_slot = pool.get<int32_t>(g.ncell);
    FMMPC_CUDA(cudaMemcpyAsync(Ls.vbv_slot, slot.data(), sizeof(int32_t) * g.ncell, cudaMemcpyHostToDevice, s));
    FMMPC_CUDA(cudaStreamSynchronize(s));
  }
  // regroup the volume-boundary lists by boundary target for the collocation pass
  {
    uint64_t *sw = tmp.get<uint64_t>(nvb + 1);
    if (nvb) k_swap_key3<<<blocks(nvb), 256, 0, s>>>(vb_k, nvb, sw);
    sort_keys(sw, nvb, 58, s, tmp);
    int32_t *ent = tmp.get<int32_t>(3 * nvb + 3);
    if (nvb) k_decode3<<<blocks(nvb), 256, 0, s>>>(sw, nvb, ent, 0);  // (level, bnd, vol)
    Ls.vbb_first = pool.get<int32_t>(g.nbcell + 1);
    Ls.vbb_src = pool.get<int32_t>(nvb + 1);
    build_csr(ent, nvb, 3, 1, 0, 1, 2, g.nbcell, Ls.vbb_first, Ls.vbb_src, s, tmp);
    uint64_t *sp = tmp.get<uint64_t>(npvb + 1);
    if (npvb) k_swap_key3<<<blocks(npvb), 256, 0, s>>>(pvb_k, npvb, sp);
    sort_keys(sp, npvb, 54, s, tmp);
    int32_t *ep = tmp.get<int32_t>(2 * npvb + 2);
    if (npvb) k_decode2<<<blocks(npvb), 256, 0, s>>>(sp, npvb, ep);  // (bnd leaf, vol leaf)
    Ls.pvb_first = pool.get<int32_t>(g.nbleaf + 1);
    Ls.pvb_src = pool.get<int32_t>(npvb + 1);
    build_csr(ep, npvb, 2, 0, -1, 0, 1, g.nbleaf, Ls.pvb_first, Ls.pvb_src, s, tmp);
  }
  FMMPC_LAUNCH_CHECK();

  // ---- host-side views: near-boundary leaves, P2P stencil
  std::vector<int32_t> pvb(2 * npvb), p2p(2 * np2p);
  if (npvb) FMMPC_CUDA(cudaMemcpyAsync(pvb.data(), Ls.p2p_vb, 8 * npvb, cudaMemcpyDeviceToHost, s));
  if (np2p) FMMPC_CUDA(cudaMemcpyAsync(p2p.data(), Ls.p2p, 8 * np2p, cudaMemcpyDeviceToHost, s));
  FMMPC_CUDA(cudaStreamSynchronize(s));
  {
    std::vector<int32_t> slot(g.nleaf, -1), first, src, leaf;
    for (int64_t e = 0; e < npvb; ++e) {
      int v = pvb[2 * e];
      if (slot[v] < 0) {
        slot[v] = (int32_t)leaf.size();
        leaf.push_back(v);
        first.push_back((int32_t)src.size());
      }
      src.push_back(pvb[2 * e + 1]);
    }
    first.push_back((int32_t)src.size());
    Ls.nbnear = (int64_t)leaf.size();
    Ls.pbv_first = pool.get<int32_t>(first.size());
    Ls.pbv_src = pool.get<int32_t>(src.size() + 1);
    Ls.pbv_leaf = pool.get<int32_t>(leaf.size() + 1);
    Ls.leaf_bslot = pool.get<int32_t>(g.nleaf);
    FMMPC_CUDA(cudaMemcpyAsync(Ls.pbv_first, first.data(), 4 * first.size(), cudaMemcpyHostToDevice, s));
    if (!src.empty()) FMMPC_CUDA(cudaMemcpyAsync(Ls.pbv_src, src.data(), 4 * src.size(), cudaMemcpyHostToDevice, s));
    if (!leaf.empty()) FMMPC_CUDA(cudaMemcpyAsync(Ls.pbv_leaf, leaf.data(), 4 * leaf.size(), cudaMemcpyHostToDevice, s));
    FMMPC_CUDA(cudaMemcpyAsync(Ls.leaf_bslot, slot.data(), 4 * g.nleaf, cudaMemcpyHostToDevice, s));
  }
  {
    // distinct leaf offsets of the P2P list; the near-field kernel sweeps them over a
    // zero-padded weight image, which is exact only if the list is the full stencil
    // clipped to the domain -- checked here.
    std::set<std::pair<int, int>> offs;
    int side = 1 << g.L;
    for (int64_t e = 0; e < np2p; ++e) {
      int tx, ty, sx, sy;
      morton_decode((uint32_t)p2p[2 * e], tx, ty);
      morton_decode((uint32_t)p2p[2 * e + 1], sx, sy);
      offs.insert({sy - ty, sx - tx});
    }
    int R = 0;
    for (auto &o : offs) R = std::max(R, std::max(std::abs(o.first), std::abs(o.second)));
    if (R > 16) throw Error(FMMPC_ERR_UNSUPPORTED, "P2P stencil radius above 16 leaves (theta too large)");
    st.R = R;
    st.count = (int)offs.size();
    for (int oy = -R; oy <= R; ++oy) {
      int lo = 1 << 20, hi = -(1 << 20), cnt = 0;
      for (auto &o : offs)
        if (o.first == oy) { lo = std::min(lo, o.second); hi = std::max(hi, o.second); ++cnt; }
      if (cnt && cnt != hi - lo + 1)
        throw Error(FMMPC_ERR_UNSUPPORTED, "P2P stencil row is not contiguous");
      st.ox0[oy + R] = cnt ? lo : 1;
      st.ox1[oy + R] = cnt ? hi : 0;
    }
    int64_t expect = 0;
    for (int ty = 0; ty < side; ++ty)
      for (int tx = 0; tx < side; ++tx)
        for (auto &o : offs) {
          int sy = ty + o.first, sx = tx + o.second;
          if (sx >= 0 && sy >= 0 && sx < side && sy < side) ++expect;
        }
    if (expect != np2p)
      throw Error(FMMPC_ERR_UNSUPPORTED, "P2P list is not a translation-invariant stencil");
  }
  FMMPC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fmmpc
