// Level-batched recursive skeletonization factorization (Sec. 2).
//
// Levels are processed leaves first (Eq. (rskelf)); every step of a level is
// one batched launch (or one launch pair per pivoted-QR step) over all boxes
// of the level:
//   A2  active DOFs I (leaf points or the children's skeletons) and the near
//       field N (active DOFs within r_near * side of the centre, Sec. 2.3.1);
//   A3  assembly of [K(N, I); K(Gamma, I)] (Eq. (proxyid)) and of the current
//       diagonal block A_II (children's X_SS, kernel entries elsewhere);
//   A4  ID by column-pivoted QR, rank k = #{j : |R_jj| > tol |R_11|},
//       T = R11^-1 R12 (Def. ID);
//   A5  X_SR = A_SR - A_SS T, X_RR = A_RR - T^T A_SR - X_SR^T T (Sec. 2.1);
//   A6  X_RR = C C^T (Sigma) or kept whole (derivative matrices,
//       Remark (indefinite)), log|F| contributions 2 sum log C_ii;
//   A7  E = X_SR X_RR^-1 and X_SS = A_SS - E X_RS;
//   A8  the root block (level 0) is factored densely.
// The host only sizes the levels (one readback of the ranks per level).
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace rsf {

// ------------------------------------------------------------ A2: I sets
struct ISeg {
  int64_t dst, src;
  int count, kind;  // kind 0: tree range (src + t), 1: copy from prev Isr
};
__global__ void build_I_kernel(const ISeg* __restrict__ segs, int nseg, const int* __restrict__ prevIsr,
                               int* __restrict__ I) {
  int sgi = blockIdx.x;
  if (sgi >= nseg) return;
  ISeg sg = segs[sgi];
  for (int t = threadIdx.x; t < sg.count; t += blockDim.x)
    I[sg.dst + t] = sg.kind ? prevIsr[sg.src + t] : (int)(sg.src + t);
}

// Near-field candidates: units are level boxes (DOFs from the level's I array)
// or coarse leaves (tree ranges).
struct Unit {
  int64_t off;
  int count, kind;  // kind 1: I[off + t], 0: off + t
};
struct NearBox {
  double cx, cy, r2;
  int u0, nu;        // unit range
  int64_t out0;      // offset of the near list
};

// Candidate units of every box of a level, on the device.  The cells of the
// box's level within ext = ceil(r_near + 1/2) cells whose square comes
// closer than r_near * w to the box centre are looked up (the box there, or
// the coarser leaf covering the cell; a coarser non-leaf means an empty
// region); each distinct box found other than the box itself is a unit.
// Boxes of one level are contiguous in breadth-first order, which is ascending
// in (set, Morton code of the cell), so a cell is found by binary search in
// its level's range of box codes.
struct NearIn {
  double cx, cy, w, lox, loy;
  int set, ix, iy, box;
};
struct BoxCodes {
  const unsigned long long* code;   // per box: set << 48 | Morton code of (ix, iy)
  const int* lev0;                  // first box of every level (L + 2 entries)
  const char* leaf;
  const int* start;
  const int* count;
  const int* level;
};
constexpr int NEAR_MAX_UNITS = 64;

__device__ __forceinline__ unsigned long long cell_code(int set, unsigned gx, unsigned gy, int lev) {
  unsigned long long c = 0;
  for (int b = lev - 1; b >= 0; b--)
    c = (c << 2) | ((unsigned long long)((gy >> b) & 1u) << 1) | (unsigned long long)((gx >> b) & 1u);
  return ((unsigned long long)set << 48) | c;
}

__device__ int find_box(const BoxCodes& K, int set, unsigned gx, unsigned gy, int lv) {
  const unsigned long long key = cell_code(set, gx, gy, lv);
  int lo = K.lev0[lv], hi = K.lev0[lv + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (K.code[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < K.lev0[lv + 1] && K.code[lo] == key) ? lo : -1;
}

// write == 0: units and candidate rows per box into nunits, ncand;
// write == 1: the units themselves from u0[i] on.
__global__ void near_units_kernel(const NearIn* __restrict__ in, int nb, int lev, double r_near, BoxCodes K,
                                  const int64_t* __restrict__ row0, const int* __restrict__ cl,
                                  int* __restrict__ nunits, int64_t* __restrict__ ncand,
                                  const int* __restrict__ u0, Unit* __restrict__ units, int write,
                                  int* __restrict__ overflow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const NearIn B = in[i];
  const double R = __dmul_rn(r_near, B.w);
  const int ext = (int)ceil(r_near + 0.5);
  const int side = 1 << lev;
  int seen[NEAR_MAX_UNITS];
  int nseen = 0, nu = 0;
  int64_t cand = 0;
  for (int dy = -ext; dy <= ext; dy++) {
    for (int dx = -ext; dx <= ext; dx++) {
      const int gx = B.ix + dx, gy = B.iy + dy;
      if (gx < 0 || gy < 0 || gx >= side || gy >= side) continue;
      const double x0 = __dadd_rn(B.lox, __dmul_rn((double)gx, B.w));
      const double y0 = __dadd_rn(B.loy, __dmul_rn((double)gy, B.w));
      const double ddx = fmax(0.0, fmax(__dsub_rn(x0, B.cx), __dsub_rn(B.cx, __dadd_rn(x0, B.w))));
      const double ddy = fmax(0.0, fmax(__dsub_rn(y0, B.cy), __dsub_rn(B.cy, __dadd_rn(y0, B.w))));
      if (__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)) >= __dmul_rn(R, R)) continue;
      int found = -1;
      for (int lv = lev; lv >= 0 && found < 0; lv--)
        found = find_box(K, B.set, (unsigned)gx >> (lev - lv), (unsigned)gy >> (lev - lv), lv);
      if (found < 0 || found == B.box) continue;
      const int flev = K.level[found];
      if (flev != lev && !K.leaf[found]) continue;   // empty region
      bool dup = false;
      for (int k = 0; k < nseen; k++) dup |= seen[k] == found;
      if (dup) continue;
      if (nseen == NEAR_MAX_UNITS) {
        atomicExch(overflow, 1);
        continue;
      }
      seen[nseen++] = found;
      Unit u;
      if (flev == lev) {
        const int fi = found - K.lev0[lev];
        u.off = row0[fi];
        u.count = cl[fi];
        u.kind = 1;
      } else {
        u.off = K.start[found];
        u.count = K.count[found];
        u.kind = 0;
      }
      if (u.count > 0) {
        if (write) units[u0[i] + nu] = u;
        nu++;
        cand += u.count;
      }
    }
  }
  if (!write) {
    nunits[i] = nu;
    ncand[i] = cand;
  }
}

// One CTA per box: ordered compaction of the candidates within the radius.
__global__ void __launch_bounds__(256) near_kernel(const NearBox* __restrict__ nbx, const Unit* __restrict__ units,
                                                   const int* __restrict__ I, const double* __restrict__ xt,
                                                   int* __restrict__ near, int* __restrict__ nnear,
                                                   QRProb* __restrict__ qp, int n_prox) {
  const NearBox B = nbx[blockIdx.x];
  __shared__ int wsum[8];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int u = B.u0; u < B.u0 + B.nu; u++) {
    const Unit U = units[u];
    for (int c0 = 0; c0 < U.count; c0 += 256) {
      int id = -1;
      int flag = 0;
      if (c0 + t < U.count) {
        id = U.kind ? I[U.off + c0 + t] : (int)(U.off + c0 + t);
        flag = dist2(xt[2 * (int64_t)id], xt[2 * (int64_t)id + 1], B.cx, B.cy) < B.r2;
      }
      unsigned m = __ballot_sync(0xffffffffu, flag);
      if (lane == 0) wsum[wid] = __popc(m);
      __syncthreads();
      int pre = 0, tot = 0;
      for (int w = 0; w < 8; w++) {
        if (w < wid) pre += wsum[w];
        tot += wsum[w];
      }
      if (flag) near[B.out0 + base + pre + __popc(m & ((1u << lane) - 1u))] = id;
      __syncthreads();
      if (t == 0) base += tot;
      __syncthreads();
    }
  }
  if (t == 0) {
    nnear[blockIdx.x] = base;
    qp[blockIdx.x].m = base + n_prox;
  }
}

// ------------------------------------------------------------ A3: assembly
struct IdBox {
  double cx, cy, w;
  int64_t row0;   // into I
  int64_t near0;  // into near
  int64_t a;      // A offset in the QR pool
  int c, lda;
};
// One warp per (box, column): rows = near field then proxy points.
__global__ void assemble_id_kernel(const IdBox* __restrict__ boxes, const int* __restrict__ colprefix,
                                   int nbox, int64_t ncols, const int* __restrict__ I,
                                   const int* __restrict__ near, const int* __restrict__ nnear,
                                   const double* __restrict__ xt, const double* __restrict__ proxy,
                                   int n_prox, KernelParams kp, double* __restrict__ pool) {
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (colprefix[mid] <= gw) lo = mid; else hi = mid - 1;
  }
  const IdBox B = boxes[lo];
  int j = (int)(gw - colprefix[lo]);
  int dj = I[B.row0 + j];
  double xj = xt[2 * (int64_t)dj], yj = xt[2 * (int64_t)dj + 1];
  int nn = nnear[lo];
  double* a = pool + B.a + (int64_t)j * B.lda;
  for (int i = lane; i < nn + n_prox; i += 32) {
    double px, py;
    if (i < nn) {
      int d = near[B.near0 + i];
      px = xt[2 * (int64_t)d]; py = xt[2 * (int64_t)d + 1];
    } else {
      int t = i - nn;
      px = B.cx + B.w * proxy[2 * t];
      py = B.cy + B.w * proxy[2 * t + 1];
    }
    a[i] = kernel_pair(kp, px, py, xj, yj);
  }
}

// Current diagonal block in [S, R] order: one warp per (box, column q).
struct AiiBox {
  int64_t row0;     // into I / perm
  int64_t aii;      // output offset (c x c, ld c)
  int c, nch, leaf, pad;
  int choff[5];     // cumulative child offsets in the local I (choff[nch] = c)
  int chld[4];      // child's c (leading dimension of its block)
  int64_t chaii[4]; // child's A_II offset in the previous pool
};
__global__ void assemble_aii_kernel(const AiiBox* __restrict__ boxes, const int* __restrict__ colprefix,
                                    int nbox, int64_t ncols, const int* __restrict__ I,
                                    const int* __restrict__ perm, const double* __restrict__ xt,
                                    KernelParams kp, const double* __restrict__ prev,
                                    double* __restrict__ out) {
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (colprefix[mid] <= gw) lo = mid; else hi = mid - 1;
  }
  const AiiBox B = boxes[lo];
  int q = (int)(gw - colprefix[lo]);
  int jl = perm[B.row0 + q];
  int dj = I[B.row0 + jl];
  double xj = xt[2 * (int64_t)dj], yj = xt[2 * (int64_t)dj + 1];
  int cj = 0, lj = jl;
  if (!B.leaf) {
    while (cj + 1 < B.nch && B.choff[cj + 1] <= jl) cj++;
    lj = jl - B.choff[cj];
  }
  double* o = out + B.aii + (int64_t)q * B.c;
  for (int p = lane; p < B.c; p += 32) {
    int il = perm[B.row0 + p];
    int di = I[B.row0 + il];
    double v;
    if (B.leaf) {
      v = (di == dj) ? kernel_diag(kp) : kernel_pair(kp, xt[2 * (int64_t)di], xt[2 * (int64_t)di + 1], xj, yj);
    } else {
      int ci = 0;
      while (ci + 1 < B.nch && B.choff[ci + 1] <= il) ci++;
      if (ci == cj) {
        int li = il - B.choff[ci];
        v = prev[B.chaii[ci] + li + (int64_t)lj * B.chld[ci]];
      } else {
        v = kernel_pair(kp, xt[2 * (int64_t)di], xt[2 * (int64_t)di + 1], xj, yj);
      }
    }
    o[p] = v;
  }
}

// Isr[row0 + p] = I[row0 + perm[row0 + p]]
__global__ void permute_I_kernel(const int* __restrict__ I, const int* __restrict__ perm,
                                 const int64_t* __restrict__ rowbox0, const int* __restrict__ rowbox,
                                 int64_t nrows, int* __restrict__ Isr) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nrows) return;
  int b = rowbox[g];
  int64_t r0 = rowbox0[b];
  Isr[g] = I[r0 + perm[g]];
}

// Gather map for the solve, then the DOF -> row map for the next level up.
__global__ void src_map_kernel(const int* __restrict__ Isr, const int* __restrict__ rowbox,
                               const char* __restrict__ leafbox, int64_t nrows,
                               const int* __restrict__ rowmap, int* __restrict__ src) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nrows) return;
  int d = Isr[g];
  src[g] = leafbox[rowbox[g]] ? -(1 + d) : rowmap[d];
}
__global__ void rowmap_kernel(const int* __restrict__ Isr, int64_t nrows, int* __restrict__ rowmap) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nrows) return;
  rowmap[Isr[g]] = (int)g;
}

// E[s, piv[i]] = t[i, s] (t: r x k column-major at t0; E: k x r at e0).
struct EScatter {
  int64_t t0, e0, col0;
  int r, k;
};
__global__ void scatter_E_kernel(const EScatter* __restrict__ es, const int64_t* __restrict__ prefix,
                                 int nprob, int64_t total, const double* __restrict__ tpool,
                                 const int* __restrict__ piv, const QRState* __restrict__ st,
                                 double* __restrict__ fpool) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const EScatter e = es[lo];
  int64_t x = g - prefix[lo];
  int i = (int)(x % e.r), s = (int)(x / e.r);
  int kq = st[lo].k;  // rank reached by the QR (r unless X_RR is singular)
  int pc = (i < kq) ? piv[e.col0 + i] : -1;
  if (i < kq) fpool[e.e0 + s + (int64_t)pc * e.k] = tpool[e.t0 + i + (int64_t)s * kq];
}

// y -= x
__global__ void axpy_neg_kernel(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y[g] -= x[g];
}

// 2 sum log diag per box (SPD levels).
struct LdBox {
  int64_t d;
  int r, slot;
};
__global__ void logdet_parts_kernel(const LdBox* __restrict__ b, int nb, const double* __restrict__ fpool,
                                    double* __restrict__ parts, DevStatus* st, int level) {
  int i = blockIdx.x;
  if (i >= nb) return;
  const LdBox B = b[i];
  __shared__ double red[256];
  double s = 0.0;
  for (int j = threadIdx.x; j < B.r; j += 256) s += log(fpool[B.d + j + (int64_t)j * B.r]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double v = 2.0 * red[0];
    if (!(v == v)) report(st, RSF_ENUMERIC, level, i, 0);
    parts[B.slot] = v;
  }
}

static void gemm(const std::vector<GemmDesc>& d, double* p0, double* p1, double* p2, cudaStream_t s) {
  if (d.empty()) return;
  GemmBatch gb;
  gb.build(d, s);
  GemmBases b{};
  b.p[0] = p0; b.p[1] = p1; b.p[2] = p2; b.p[3] = nullptr;
  b.sc[0] = b.sc[1] = b.sc[2] = b.sc[3] = 1;
  b.alpha_scale = 1.0;
  gb.run(b, s);
}

static GemmDesc gd(int M, int N, int K, int8_t abase, int64_t a, int lda, int8_t ta, int8_t bbase, int64_t b,
                   int ldb, int8_t tb, int8_t cbase, int64_t c, int ldc, double alpha, double beta,
                   int8_t triB = 0, int8_t lowC = 0) {
  GemmDesc g{};
  g.M = M; g.N = N; g.K = K;
  g.abase = abase; g.a = a; g.lda = lda; g.ta = ta;
  g.bbase = bbase; g.b = b; g.ldb = ldb; g.tb = tb;
  g.cbase = cbase; g.c = c; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta; g.triB = triB; g.lowC = lowC;
  return g;
}

static std::vector<double> proxy_table(const rsf_opts& o) {
  // unit offsets of the proxy annulus (multiply by the box side)
  std::vector<double> t;
  int n_ang = o.n_prox / o.n_rings;
  for (int i = 0; i < o.n_rings; i++) {
    double rad = o.r_in + (o.r_out - o.r_in) * (i + 0.5) / o.n_rings;
    double off = (i % 2) ? 0.5 : 0.0;
    for (int a = 0; a < n_ang; a++) {
      double ang = 2.0 * M_PI * (a + off) / n_ang;
      t.push_back(rad * std::cos(ang));
      t.push_back(rad * std::sin(ang));
    }
  }
  return t;
}

void factorize(rsf_handle_s* h) {
  TreeData& T = h->tree_raw->t;
  const rsf_opts& o = h->opts;
  cudaStream_t s = h->stream;
  const KernelParams kp = h->kp;
  const int L = T.L;
  const int64_t n = T.n;
  const int nboxes = (int)T.level.size();
  RSF_CHECK(o.n_prox >= 0 && o.n_rings >= 1 && o.n_prox % o.n_rings == 0, RSF_EINVAL,
            "n_prox must be a multiple of n_rings");
  h->levels.clear();
  h->levels.resize(L + 1);
  h->status.alloc(sizeof(DevStatus), s);
  h->status.zero();
  DevStatus* dst = h->status.as<DevStatus>();
  h->logdet_parts.alloc(sizeof(double) * nboxes, s);
  h->logdet_parts.zero();
  h->nboxes_total = nboxes;

  std::vector<double> ptab = proxy_table(o);
  DBuf dproxy;
  upload(dproxy, ptab, s);
  DBuf rowmap;
  rowmap.alloc(sizeof(int) * n, s);
  // box codes for the device near-field lookup (boxes of different point
  // sets are never neighbours: the set sits above the cell code)
  DBuf dcode, dlev0, dbleaf, dbstart, dbcount, dblevel;
  {
    std::vector<unsigned long long> code(nboxes);
    std::vector<int> lev0(L + 2, 0);
    for (int b = 0; b < nboxes; b++) {
      unsigned long long c = 0;
      for (int bit = T.level[b] - 1; bit >= 0; bit--)
        c = (c << 2) | ((unsigned long long)((T.iy[b] >> bit) & 1) << 1) | (unsigned long long)((T.ix[b] >> bit) & 1);
      code[b] = ((unsigned long long)T.box_set[b] << 48) | c;
      lev0[T.level[b] + 1]++;
    }
    for (int l = 0; l <= L; l++) lev0[l + 1] += lev0[l];
    for (int l = 0; l <= L; l++)
      RSF_CHECK(T.by_level[l].empty() || (T.by_level[l].front() == lev0[l] && T.by_level[l].back() == lev0[l + 1] - 1),
                RSF_ECUDA, "box table: levels are not contiguous");
    for (int b = 1; b < nboxes; b++)
      RSF_CHECK(T.level[b] != T.level[b - 1] || code[b] > code[b - 1], RSF_ECUDA,
                "box table: a level is not in ascending cell order");
    std::vector<char> leafv(T.is_leaf.begin(), T.is_leaf.end());
    upload(dcode, code, s);
    upload(dlev0, lev0, s);
    upload(dbleaf, leafv, s);
    upload(dbstart, T.start, s);
    upload(dbcount, T.count, s);
    upload(dblevel, T.level, s);
  }
  const BoxCodes bcodes{dcode.as<unsigned long long>(), dlev0.as<int>(), dbleaf.as<char>(), dbstart.as<int>(),
                        dbcount.as<int>(), dblevel.as<int>()};

  std::vector<int> box2idx(nboxes, -1);   // index of a box within its level
  DBuf prevAII;                           // A_II pool of the level below (children's X_SS)
  std::vector<int64_t> prevAIIoff;        // per box of the level below
  const int* prevIsr = nullptr;
  double flops = 0, kevals = 0;
  int64_t fentries = 0;
  int max_rank = 0, max_active = 0;

  for (int lev = L; lev >= 0; lev--) {
    LevelData& Lv = h->levels[lev];
    Lv.lev = lev;
    Lv.box = T.by_level[lev];
    const int nb = (int)Lv.box.size();
    Lv.nb = nb;
    for (int i = 0; i < nb; i++) box2idx[Lv.box[i]] = i;
    LevelData* child = (lev < L) ? &h->levels[lev + 1] : nullptr;
    // ---- sizes and I sets
    Lv.c.assign(nb, 0);
    Lv.leafbox.assign(nb, 0);
    std::vector<ISeg> segs;
    Lv.row0.assign(nb + 1, 0);
    for (int i = 0; i < nb; i++) {
      int b = Lv.box[i];
      Lv.leafbox[i] = T.is_leaf[b];
      if (T.is_leaf[b]) {
        Lv.c[i] = T.count[b];
      } else {
        int c = 0;
        for (int sl = 0; sl < 4; sl++) {
          int cb = T.children[b][sl];
          if (cb >= 0) c += child->k[box2idx[cb]];
        }
        Lv.c[i] = c;
      }
      Lv.row0[i + 1] = Lv.row0[i] + Lv.c[i];
    }
    Lv.nrows = Lv.row0[nb];
    for (int i = 0; i < nb; i++) {
      int b = Lv.box[i];
      if (T.is_leaf[b]) {
        segs.push_back({Lv.row0[i], (int64_t)T.start[b], T.count[b], 0});
      } else {
        int64_t dst0 = Lv.row0[i];
        for (int sl = 0; sl < 4; sl++) {
          int cb = T.children[b][sl];
          if (cb < 0) continue;
          int ci = box2idx[cb];
          int kc = child->k[ci];
          if (kc > 0) segs.push_back({dst0, child->row0[ci], kc, 1});
          dst0 += kc;
        }
      }
      max_active = std::max(max_active, Lv.c[i]);
    }
    DBuf I;
    I.alloc(sizeof(int) * std::max<int64_t>(1, Lv.nrows), s);
    {
      DBuf dseg;
      upload(dseg, segs, s);
      LAUNCH(build_I_kernel, (int)segs.size(), 128, 0, s, dseg.as<ISeg>(), (int)segs.size(), prevIsr,
             I.as<int>());
    }
    std::vector<int> rowbox(Lv.nrows);
    for (int i = 0; i < nb; i++)
      for (int64_t r = Lv.row0[i]; r < Lv.row0[i + 1]; r++) rowbox[r] = i;
    DBuf drowbox, drow0, dleaf, dcl;
    upload(drowbox, rowbox, s);
    upload(drow0, Lv.row0, s);
    upload(dleaf, Lv.leafbox, s);
    upload(dcl, Lv.c, s);

    // ---- ID (A2-A4), skipped at the root
    Lv.k.assign(nb, 0);
    DBuf perm;
    perm.alloc(sizeof(int) * std::max<int64_t>(1, Lv.nrows), s);
    std::vector<int64_t> Toff(nb, 0);
    QRBatch qb;
    DBuf qrpool, near, nnear;
    if (lev > 0) {
      // near-field candidate units, enumerated on the device
      std::vector<NearBox> nbx(nb);
      std::vector<int64_t> cand(nb, 0);
      int64_t near_total = 0;
      DBuf dunits;
      {
        std::vector<NearIn> nin(nb);
        for (int i = 0; i < nb; i++) {
          const int b = Lv.box[i], bs = T.box_set[b];
          nin[i] = NearIn{T.cx[b], T.cy[b], T.w[b], T.set_lo[2 * bs], T.set_lo[2 * bs + 1], bs, T.ix[b], T.iy[b], b};
        }
        DBuf dnin, dnu, dcand, du0, dovf;
        upload(dnin, nin, s);
        dnu.alloc(sizeof(int) * nb, s);
        dcand.alloc(sizeof(int64_t) * nb, s);
        dovf.alloc(sizeof(int), s);
        dovf.zero();
        LAUNCH(near_units_kernel, cdiv(nb, 128), 128, 0, s, dnin.as<NearIn>(), nb, lev, o.r_near, bcodes,
               drow0.as<int64_t>(), dcl.as<int>(), dnu.as<int>(), dcand.as<int64_t>(), nullptr, nullptr, 0,
               dovf.as<int>());
        std::vector<int> nu(nb);
        int ovf = 0;
        d2h(nu.data(), dnu.as<int>(), nb, s);
        d2h(cand.data(), dcand.as<int64_t>(), nb, s);
        d2h(&ovf, dovf.as<int>(), 1, s);
        sync(s);
        RSF_CHECK(!ovf, RSF_EINVAL, "near field: too many neighbour boxes (r_near too large)");
        std::vector<int> u0(nb + 1, 0);
        for (int i = 0; i < nb; i++) {
          u0[i + 1] = u0[i] + nu[i];
          nbx[i].cx = T.cx[Lv.box[i]];
          nbx[i].cy = T.cy[Lv.box[i]];
          const double R = o.r_near * T.w[Lv.box[i]];
          nbx[i].r2 = R * R;
          nbx[i].u0 = u0[i];
          nbx[i].nu = nu[i];
          nbx[i].out0 = near_total;
          near_total += cand[i];
        }
        upload(du0, u0, s);
        dunits.alloc(sizeof(Unit) * std::max(1, u0[nb]), s);
        LAUNCH(near_units_kernel, cdiv(nb, 128), 128, 0, s, dnin.as<NearIn>(), nb, lev, o.r_near, bcodes,
               drow0.as<int64_t>(), dcl.as<int>(), nullptr, nullptr, du0.as<int>(), dunits.as<Unit>(), 1,
               dovf.as<int>());
      }
      // QR problems: A = [near; proxy] x c, ld = cand + n_prox
      std::vector<QRProb> qp(nb);
      std::vector<IdBox> idb(nb);
      std::vector<int> colpre(nb + 1, 0);
      int64_t apool = 0;
      for (int i = 0; i < nb; i++) {
        int b = Lv.box[i];
        int ld = (int)(cand[i] + o.n_prox);
        qp[i].m = ld;  // upper bound; the near kernel writes the true count
        qp[i].c = Lv.c[i];
        qp[i].cpiv = Lv.c[i];
        qp[i].maxk = Lv.c[i];
        qp[i].lda = std::max(1, ld);
        qp[i].a = apool;
        qp[i].tol = h->tol;
        idb[i] = {T.cx[b], T.cy[b], T.w[b], Lv.row0[i], nbx[i].out0, apool, Lv.c[i], std::max(1, ld)};
        apool += (int64_t)std::max(1, ld) * Lv.c[i];
        colpre[i + 1] = colpre[i] + Lv.c[i];
      }
      qb.build(qp, s);
      near.alloc(sizeof(int) * std::max<int64_t>(1, near_total), s);
      nnear.alloc(sizeof(int) * nb, s);
      {
        DBuf dnbx;
        upload(dnbx, nbx, s);
        LAUNCH(near_kernel, nb, 256, 0, s, dnbx.as<NearBox>(), dunits.as<Unit>(), I.as<int>(),
               T.xt.as<double>(), near.as<int>(), nnear.as<int>(), qb.d_prob(), o.n_prox);
      }
      qrpool.alloc(sizeof(double) * std::max<int64_t>(1, apool), s);
      {
        DBuf didb, dcol;
        upload(didb, idb, s);
        upload(dcol, colpre, s);
        LAUNCH(assemble_id_kernel, cdiv((int64_t)colpre[nb] * 32, 256), 256, 0, s, didb.as<IdBox>(),
               dcol.as<int>(), nb, (int64_t)colpre[nb], I.as<int>(), near.as<int>(), nnear.as<int>(),
               T.xt.as<double>(), dproxy.as<double>(), o.n_prox, kp, qrpool.as<double>());
      }
      qb.run(qrpool.as<double>(), dst, lev, s);
      DBuf dkout;
      dkout.alloc(sizeof(int) * nb, s);
      qr_split(qb, drow0.as<int64_t>(), perm.as<int>(), dkout.as<int>(), s);
      d2h(Lv.k.data(), dkout.as<int>(), nb, s);
      std::vector<int> hnn(nb);
      d2h(hnn.data(), nnear.as<int>(), nb, s);
      sync(s);
      for (int i = 0; i < nb; i++) {
        double m = hnn[i] + o.n_prox, c = Lv.c[i], k = Lv.k[i];
        kevals += m * c;
        flops += 4.0 * m * c * k - 2.0 * k * k * (m + c) + 4.0 * k * k * k / 3.0;
      }
    } else {
      // root: no ID; every remaining DOF stays in its dense block (k = 0).
      std::vector<int> idp(Lv.nrows);
      for (int i = 0; i < nb; i++)
        for (int64_t r = Lv.row0[i]; r < Lv.row0[i + 1]; r++) idp[r] = (int)(r - Lv.row0[i]);
      h2d(perm.as<int>(), idp.data(), idp.size(), s);
    }
    Lv.r.assign(nb, 0);
    for (int i = 0; i < nb; i++) {
      Lv.r[i] = Lv.c[i] - Lv.k[i];
      max_rank = std::max(max_rank, Lv.k[i]);
    }
    // ---- [S, R]-ordered DOF list and solve maps
    Lv.Isr.alloc(sizeof(int) * std::max<int64_t>(1, Lv.nrows), s);
    LAUNCH(permute_I_kernel, cdiv(Lv.nrows, 256), 256, 0, s, I.as<int>(), perm.as<int>(), drow0.as<int64_t>(),
           drowbox.as<int>(), Lv.nrows, Lv.Isr.as<int>());
    Lv.src.alloc(sizeof(int) * std::max<int64_t>(1, Lv.nrows), s);
    LAUNCH(src_map_kernel, cdiv(Lv.nrows, 256), 256, 0, s, Lv.Isr.as<int>(), drowbox.as<int>(),
           dleaf.as<char>(), Lv.nrows, rowmap.as<int>(), Lv.src.as<int>());
    LAUNCH(rowmap_kernel, cdiv(Lv.nrows, 256), 256, 0, s, Lv.Isr.as<int>(), Lv.nrows, rowmap.as<int>());

    // ---- factor pool layout
    Lv.toff.assign(nb, 0); Lv.eoff.assign(nb, 0); Lv.doff.assign(nb, 0); Lv.dioff.assign(nb, 0);
    int64_t fp = 0;
    for (int i = 0; i < nb; i++) {
      int64_t k = Lv.k[i], r = Lv.r[i];
      Lv.toff[i] = fp; fp += k * r;
      Lv.eoff[i] = fp; fp += k * r;
      Lv.doff[i] = fp; fp += r * r;
      if (h->spd) { Lv.dioff[i] = fp; fp += r * r; }
    }
    Lv.fpool.alloc(sizeof(double) * std::max<int64_t>(1, fp), s);
    Lv.fpool.zero();
    double* F = Lv.fpool.as<double>();
    for (int i = 0; i < nb; i++) fentries += 2 * (int64_t)Lv.k[i] * Lv.r[i] + (int64_t)Lv.r[i] * Lv.r[i];

    // ---- T = R11^-1 R12 (A4)
    if (lev > 0) {
      std::vector<TrsmProb> tp(nb);
      for (int i = 0; i < nb; i++) {
        tp[i].nrhs = Lv.k[i] > 0 ? Lv.r[i] : 0;
        tp[i].rhs0 = Lv.row0[i] + Lv.k[i];
        tp[i].out0 = Lv.toff[i];
        flops += (double)Lv.k[i] * Lv.k[i] * Lv.r[i];
      }
      qr_trsm(qb, tp, perm.as<int>(), qrpool.as<double>(), F, dst, lev, s);
    }
    qrpool.release();
    near.release();

    // ---- current diagonal block A_II in [S, R] order (A3)
    std::vector<AiiBox> ab(nb);
    std::vector<int64_t> aiioff(nb + 1, 0);
    std::vector<int> colpre(nb + 1, 0);
    for (int i = 0; i < nb; i++) {
      int b = Lv.box[i];
      AiiBox& B = ab[i];
      B = AiiBox{};
      B.row0 = Lv.row0[i];
      B.aii = aiioff[i];
      B.c = Lv.c[i];
      B.leaf = T.is_leaf[b];
      B.nch = 0;
      int off = 0;
      if (!B.leaf) {
        for (int sl = 0; sl < 4; sl++) {
          int cb = T.children[b][sl];
          if (cb < 0) continue;
          int ci = box2idx[cb];
          B.choff[B.nch] = off;
          B.chld[B.nch] = child->c[ci];
          B.chaii[B.nch] = prevAIIoff[ci];
          off += child->k[ci];
          B.nch++;
        }
        B.choff[B.nch] = off;
      }
      aiioff[i + 1] = aiioff[i] + (int64_t)Lv.c[i] * Lv.c[i];
      colpre[i + 1] = colpre[i] + Lv.c[i];
      kevals += (double)Lv.c[i] * Lv.c[i];
    }
    DBuf AII;
    AII.alloc(sizeof(double) * std::max<int64_t>(1, aiioff[nb]), s);
    {
      DBuf dab, dcol;
      upload(dab, ab, s);
      upload(dcol, colpre, s);
      LAUNCH(assemble_aii_kernel, cdiv((int64_t)colpre[nb] * 32, 256), 256, 0, s, dab.as<AiiBox>(),
             dcol.as<int>(), nb, (int64_t)colpre[nb], I.as<int>(), perm.as<int>(), T.xt.as<double>(), kp,
             prevAII.as<double>(), AII.as<double>());
    }
    double* A = AII.as<double>();

    // ---- transform (A5): C base 0 = AII, 2 = factor pool
    {
      std::vector<GemmDesc> g1, g2, g3;
      for (int i = 0; i < nb; i++) {
        int c = Lv.c[i], k = Lv.k[i], r = Lv.r[i];
        if (k == 0 || r == 0) continue;
        int64_t a0 = aiioff[i];
        int64_t SS = a0, SR = a0 + (int64_t)k * c, RR = a0 + k + (int64_t)k * c;
        // X_RR -= T^T A_SR
        g1.push_back(gd(r, r, k, 2, Lv.toff[i], k, 1, 0, SR, c, 0, 0, RR, c, -1.0, 1.0));
        // X_SR = A_SR - A_SS T
        g2.push_back(gd(k, r, k, 0, SS, c, 0, 2, Lv.toff[i], k, 0, 0, SR, c, -1.0, 1.0));
        // X_RR -= X_SR^T T
        g3.push_back(gd(r, r, k, 0, SR, c, 1, 2, Lv.toff[i], k, 0, 0, RR, c, -1.0, 1.0));
        flops += 2.0 * k * k * r + 4.0 * k * r * r;
      }
      gemm(g1, A, nullptr, F, s);
      gemm(g2, A, nullptr, F, s);
      gemm(g3, A, nullptr, F, s);
      std::vector<SqProb> sq;
      for (int i = 0; i < nb; i++)
        if (Lv.r[i] > 0) sq.push_back({Lv.r[i], Lv.c[i], aiioff[i] + Lv.k[i] + (int64_t)Lv.k[i] * Lv.c[i]});
      symmetrize_batched(sq, A, s);
    }

    // ---- diagonal factor (A6) and Schur update (A7)
    {
      std::vector<CopyProb> cp;
      for (int i = 0; i < nb; i++) {
        int c = Lv.c[i], k = Lv.k[i], r = Lv.r[i];
        if (r == 0) continue;
        cp.push_back({r, r, c, r, aiioff[i] + k + (int64_t)k * c, Lv.doff[i], 0});
      }
      copy_batched(cp, A, F, s);
    }
    if (h->spd) {
      std::vector<CholProb> ch;
      std::vector<TriInvProb> ti;
      for (int i = 0; i < nb; i++) {
        if (Lv.r[i] == 0) continue;
        ch.push_back({Lv.r[i], Lv.r[i], Lv.doff[i], Lv.box[i]});
        ti.push_back({Lv.r[i], Lv.r[i], Lv.doff[i], Lv.dioff[i]});
        flops += std::pow((double)Lv.r[i], 3) / 3.0 * 2.0;
      }
      cholesky_batched(ch, F, dst, lev, s);
      lower_inverse_batched(ti, F, F, s);
      // V = X_SR Cinv^T (temp), X_SS = A_SS - V V^T, E = V Cinv
      std::vector<int64_t> voff(nb + 1, 0);
      for (int i = 0; i < nb; i++) voff[i + 1] = voff[i] + (int64_t)Lv.k[i] * Lv.r[i];
      DBuf V;
      V.alloc(sizeof(double) * std::max<int64_t>(1, voff[nb]), s);
      std::vector<GemmDesc> g1, g2, g3;
      for (int i = 0; i < nb; i++) {
        int c = Lv.c[i], k = Lv.k[i], r = Lv.r[i];
        if (k == 0 || r == 0) continue;
        int64_t a0 = aiioff[i];
        int64_t SS = a0, SR = a0 + (int64_t)k * c;
        g1.push_back(gd(k, r, r, 0, SR, c, 0, 2, Lv.dioff[i], r, 1, 1, voff[i], k, 1.0, 0.0, 2));
        g2.push_back(gd(k, k, r, 1, voff[i], k, 0, 1, voff[i], k, 1, 0, SS, c, -1.0, 1.0));
        g3.push_back(gd(k, r, r, 1, voff[i], k, 0, 2, Lv.dioff[i], r, 0, 2, Lv.eoff[i], k, 1.0, 0.0, 1));
        flops += 2.0 * k * r * r + 2.0 * k * k * r;
      }
      gemm(g1, A, V.as<double>(), F, s);
      gemm(g2, A, V.as<double>(), F, s);
      gemm(g3, A, V.as<double>(), F, s);
      // log-determinant pieces
      std::vector<LdBox> ld;
      for (int i = 0; i < nb; i++)
        if (Lv.r[i] > 0) ld.push_back({Lv.doff[i], Lv.r[i], Lv.box[i]});
      if (!ld.empty()) {
        DBuf dld;
        upload(dld, ld, s);
        LAUNCH(logdet_parts_kernel, (int)ld.size(), 256, 0, s, dld.as<LdBox>(), (int)ld.size(), F,
               h->logdet_parts.as<double>(), dst, lev);
      }
    } else if (lev > 0) {
      // E^T = X_RR^-1 X_RS by pivoted QR of [X_RR | X_RS] and back-substitution
      std::vector<QRProb> qp;
      std::vector<int> idx;
      std::vector<CopyProb> cp;
      int64_t qpool = 0;
      for (int i = 0; i < nb; i++) {
        int c = Lv.c[i], k = Lv.k[i], r = Lv.r[i];
        if (k == 0 || r == 0) continue;
        QRProb q{};
        q.m = r; q.c = r + k; q.cpiv = r; q.maxk = r; q.lda = r; q.a = qpool; q.tol = 0.0;
        int64_t a0 = aiioff[i];
        cp.push_back({r, r, c, r, a0 + k + (int64_t)k * c, qpool, 0});                  // X_RR
        cp.push_back({r, k, c, r, a0 + (int64_t)k * c, qpool + (int64_t)r * r, 1});     // X_RS = X_SR^T
        qpool += (int64_t)r * (r + k);
        qp.push_back(q);
        idx.push_back(i);
        flops += 4.0 / 3.0 * std::pow((double)r, 3) + 2.0 * (double)r * r * k + (double)r * r * k;
      }
      if (!qp.empty()) {
        DBuf qpm;
        qpm.alloc(sizeof(double) * qpool, s);
        copy_batched(cp, A, qpm.as<double>(), s);
        QRBatch qe;
        qe.build(qp, s);
        qe.run(qpm.as<double>(), dst, lev, s);
        std::vector<int> rhs;
        std::vector<TrsmProb> tp(qp.size());
        int64_t tout = 0;
        std::vector<EScatter> es(qp.size());
        std::vector<int64_t> epre(qp.size() + 1, 0);
        for (size_t j = 0; j < qp.size(); j++) {
          int i = idx[j];
          int r = Lv.r[i], k = Lv.k[i];
          tp[j].nrhs = k;
          tp[j].rhs0 = (int64_t)rhs.size();
          tp[j].out0 = tout;
          for (int t = 0; t < k; t++) rhs.push_back(r + t);
          es[j] = {tout, Lv.eoff[i], qe.colprefix_h[j], r, k};
          tout += (int64_t)r * k;
          epre[j + 1] = epre[j] + (int64_t)r * k;
        }
        DBuf drhs, tpoolb;
        upload(drhs, rhs, s);
        tpoolb.alloc(sizeof(double) * std::max<int64_t>(1, tout), s);
        qr_trsm(qe, tp, drhs.as<int>(), qpm.as<double>(), tpoolb.as<double>(), dst, lev, s);
        DBuf des, dep;
        upload(des, es, s);
        upload(dep, epre, s);
        LAUNCH(scatter_E_kernel, cdiv(epre.back(), 256), 256, 0, s, des.as<EScatter>(), dep.as<int64_t>(),
               (int)es.size(), epre.back(), tpoolb.as<double>(), qe.d_piv(), qe.d_state(), F);
        // X_SS = A_SS - E X_RS
        std::vector<GemmDesc> g;
        for (int i = 0; i < nb; i++) {
          int c = Lv.c[i], k = Lv.k[i], r = Lv.r[i];
          if (k == 0 || r == 0) continue;
          int64_t a0 = aiioff[i];
          g.push_back(gd(k, k, r, 2, Lv.eoff[i], k, 0, 0, a0 + (int64_t)k * c, c, 1, 0, a0, c, -1.0, 1.0));
          flops += 2.0 * k * k * r;
        }
        gemm(g, A, nullptr, F, s);
      }
    }
    {
      std::vector<SqProb> sq;
      for (int i = 0; i < nb; i++)
        if (Lv.k[i] > 0) sq.push_back({Lv.k[i], Lv.c[i], aiioff[i]});
      symmetrize_batched(sq, A, s);
    }

    // ---- solve descriptors for this level (bases: 0 = X, 1 = tmp, 2 = fpool)
    {
      std::vector<GemmDesc> rsT, srE, rsE, srT;
      std::vector<GemmDesc> mid[5];
      std::vector<int64_t> rr;
      Lv.boxRSE.clear();
      for (int v = 0; v < 5; v++) Lv.boxMid[v].clear();
      for (int i = 0; i < nb; i++) {
        int k = Lv.k[i], r = Lv.r[i];
        int64_t S0 = Lv.row0[i], R0 = Lv.row0[i] + k;
        if (k > 0 && r > 0) {
          Lv.boxRSE.push_back(i);
          // row block offsets are rows * ld with ld = q: stored as rows, scaled at launch
          rsT.push_back(gd(-1, r, k, 0, S0, -1, 0, 2, Lv.toff[i], k, 0, 0, R0, -1, 1.0, 1.0));
          srE.push_back(gd(-1, k, r, 0, R0, -1, 0, 2, Lv.eoff[i], k, 1, 0, S0, -1, 1.0, 1.0));
          rsE.push_back(gd(-1, r, k, 0, S0, -1, 0, 2, Lv.eoff[i], k, 0, 0, R0, -1, 1.0, 1.0));
          srT.push_back(gd(-1, k, r, 0, R0, -1, 0, 2, Lv.toff[i], k, 1, 0, S0, -1, 1.0, 1.0));
        }
        if (r > 0) {
          for (int v = 0; v < 5; v++)
            if ((v < 4) == h->spd) Lv.boxMid[v].push_back(i);
          if (h->spd) {
            mid[0].push_back(gd(-1, r, r, 0, R0, -1, 0, 2, Lv.dioff[i], r, 1, 1, R0, -1, 1.0, 0.0, 2));
            mid[1].push_back(gd(-1, r, r, 0, R0, -1, 0, 2, Lv.dioff[i], r, 0, 1, R0, -1, 1.0, 0.0, 1));
            mid[2].push_back(gd(-1, r, r, 0, R0, -1, 0, 2, Lv.doff[i], r, 0, 1, R0, -1, 1.0, 0.0, 1));
            mid[3].push_back(gd(-1, r, r, 0, R0, -1, 0, 2, Lv.doff[i], r, 1, 1, R0, -1, 1.0, 0.0, 2));
          } else {
            mid[4].push_back(gd(-1, r, r, 0, R0, -1, 0, 2, Lv.doff[i], r, 0, 1, R0, -1, 1.0, 0.0, 0));
          }
          rr.push_back(R0);
          rr.push_back(r);
        }
      }
      Lv.gRS_T.build(rsT, s);
      Lv.gSR_Et.build(srE, s);
      Lv.gRS_E.build(rsE, s);
      Lv.gSR_Tt.build(srT, s);
      for (int v = 0; v < 5; v++) Lv.gMid[v].build(mid[v], s);
      Lv.hRS_T = std::move(rsT);
      Lv.hSR_Et = std::move(srE);
      Lv.hRS_E = std::move(rsE);
      Lv.hSR_Tt = std::move(srT);
      for (int v = 0; v < 5; v++) Lv.hMid[v] = std::move(mid[v]);
      Lv.nrr = (int)rr.size() / 2;
      upload(Lv.rr, rr, s);
    }

    // keep this level's A_II (its X_SS blocks) for the parent level
    prevAII = std::move(AII);
    prevAIIoff.assign(aiioff.begin(), aiioff.end() - 1);
    prevIsr = Lv.Isr.as<int>();
    sync(s);  // host vectors used by uploads above stay valid until here
  }
  // mixed precision: the solve factors are used as df64 pairs from here on
  if (h->df) {
    if (h->spd) {
      for (auto& Lv : h->levels) convert_df64(Lv.fpool.as<double>(), (int64_t)(Lv.fpool.bytes / sizeof(double)), 1, s);
    } else {
      // A derivative matrix is eliminated with indefinite diagonal blocks,
      // which can amplify rounding errors far beyond the ID tolerance.  Probe
      // one application in fp64 and in df64 and keep df64 when the two agree
      // to DF64_APPLY_TOL_FACTOR x the ID tolerance.  F_l feeds only the
      // quadratic term alpha^T F_l alpha and the peeled trace of
      // (F^-1 F_l + F_l F^-1)/2 (Algorithm 1); a relative apply error delta
      // moves both by about delta of their size, and Sec. 5.3 pairs
      // eps_fact with eps_peel = 1000 eps_fact, so 10 eps_fact keeps the
      // rounding two orders of magnitude below the peeling error of the
      // trace and of the same order as the factorization's own error.
      const int form = h->df;
      h->df = 0;
      std::vector<double> hx(n);
      uint64_t st = 0x9E3779B97F4A7C15ull;
      for (int64_t i = 0; i < n; i++) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        hx[i] = (double)(int64_t)(st >> 11) / 9007199254740992.0 - 0.5;
      }
      DBuf x, y64, ydf;
      upload(x, hx, s);
      y64.alloc(sizeof(double) * n, s);
      ydf.alloc(sizeof(double) * n, s);
      solve_rows(h, RSF_OP_APPLY, x.as<double>(), y64.as<double>(), 1, 0);
      std::vector<DBuf> keep(h->levels.size());
      for (size_t l = 0; l < h->levels.size(); l++) {
        LevelData& Lv = h->levels[l];
        DBuf c;
        c.alloc(Lv.fpool.bytes, s);
        if (Lv.fpool.bytes) RSF_CUDA(cudaMemcpyAsync(c.p, Lv.fpool.p, Lv.fpool.bytes, cudaMemcpyDeviceToDevice, s));
        convert_df64(c.as<double>(), (int64_t)(c.bytes / sizeof(double)), 1, s);
        keep[l] = std::move(Lv.fpool);
        Lv.fpool = std::move(c);
      }
      h->df = form;
      solve_rows(h, RSF_OP_APPLY, x.as<double>(), ydf.as<double>(), 1, 0);
      double nn = dot_device(y64.as<double>(), y64.as<double>(), n, s);
      LAUNCH(axpy_neg_kernel, cdiv(n, 256), 256, 0, s, ydf.as<double>(), y64.as<double>(), n);
      double dd = dot_device(ydf.as<double>(), ydf.as<double>(), n, s);
      const double lim = DF64_APPLY_TOL_FACTOR * h->tol;
      bool ok = std::isfinite(dd) && dd <= lim * lim * nn;
      h->probe_rel_diff = std::sqrt(dd / std::max(nn, 1e-300));
      if (verbose())
        fprintf(stderr, "[rsf] derivative factorization: df64 vs fp64 apply rel diff %.3e -> %s\n",
                std::sqrt(dd / std::max(nn, 1e-300)), ok ? "df64" : "fp64");
      if (!ok) {
        for (size_t l = 0; l < h->levels.size(); l++) h->levels[l].fpool = std::move(keep[l]);
        h->df = 0;
      }
    }
  }
  h->flops = flops;
  h->kevals = kevals;
  h->factor_entries = fentries;
  h->max_rank = max_rank;
  h->max_active = max_active;
}

void check_status(rsf_handle_s* h) {
  DevStatus st{};
  d2h(&st, h->status.as<DevStatus>(), 1, h->stream);
  sync(h->stream);
  const int tcs = tc_status_take();
  if (tcs != 0) fail((rsf_status)tcs, "tensor-core GEMM: a bounded wait gave up");
  if (st.code != 0) {
    char buf[160];
    snprintf(buf, sizeof buf, "device status %d at level %d box %d (detail %d)", st.code, st.level, st.box,
             st.detail);
    fail((rsf_status)st.code, buf);
  }
}

}  // namespace rsf
