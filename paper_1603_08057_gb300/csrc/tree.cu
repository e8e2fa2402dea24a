// Quadtree construction (Sec. 2.1, Remark (tree)), all on the device.
//
// Bounding box reduction, quantised coordinates and Morton keys (D = 24 bits
// per axis, y bit above x bit, so child slots are SW, SE, NW, NE), a stable
// least-significant-digit radix sort of (key, index) written here (8-bit
// digits; ties keep the original index order), the gather of the coordinates
// into tree order, and the box table: a breadth-first split of every box that
// holds more than n_occ points, by binary searches of its children's key
// ranges, in one single-CTA kernel.  The host receives the finished table
// (O(n / n_occ) boxes), which it needs to size every level.
//
// A forest of independent point sets (batched datasets) is built the same
// way: every set gets its own root square, its set index sits above the 48
// Morton bits of the key, so one radix sort groups the sets (in order) and
// orders each set's points; every box records its set.  Boxes of different
// sets never interact.
#include <algorithm>
#include <array>
#include <cmath>

#include "internal.cuh"

namespace rsf {

__global__ void bbox_partial_kernel(const double* __restrict__ pts, int64_t n, double* __restrict__ part) {
  __shared__ double s[4][256];
  double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = pts[2 * i], y = pts[2 * i + 1];
    mnx = fmin(mnx, x); mxx = fmax(mxx, x); mny = fmin(mny, y); mxy = fmax(mxy, y);
  }
  int t = threadIdx.x;
  s[0][t] = mnx; s[1][t] = mxx; s[2][t] = mny; s[3][t] = mxy;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
      s[0][t] = fmin(s[0][t], s[0][t + o]); s[1][t] = fmax(s[1][t], s[1][t + o]);
      s[2][t] = fmin(s[2][t], s[2][t + o]); s[3][t] = fmax(s[3][t], s[3][t + o]);
    }
    __syncthreads();
  }
  if (t == 0) {
    part[4 * blockIdx.x + 0] = s[0][0]; part[4 * blockIdx.x + 1] = s[1][0];
    part[4 * blockIdx.x + 2] = s[2][0]; part[4 * blockIdx.x + 3] = s[3][0];
  }
}

// Set of tree position / point i: the last set whose offset is <= i.
__device__ __forceinline__ int set_of(const int64_t* __restrict__ off, int nsets, int64_t i) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void keys_kernel(const double* __restrict__ pts, int64_t n, const int64_t* __restrict__ set_off,
                            int nsets, const double* __restrict__ set_geom, unsigned long long* __restrict__ keys,
                            int* __restrict__ idx, int* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sidx = set_of(set_off, nsets, i);
  const double lox = set_geom[3 * sidx], loy = set_geom[3 * sidx + 1], scale = set_geom[3 * sidx + 2];
  const double qmax = (double)((1u << DEPTH_BITS) - 1u);
  double x = pts[2 * i], y = pts[2 * i + 1];
  if (!(x == x) || !(y == y) || fabs(x) > 1e300 || fabs(y) > 1e300) atomicExch(bad, 1);
  double fx = floor(__dmul_rn(__dsub_rn(x, lox), scale));
  double fy = floor(__dmul_rn(__dsub_rn(y, loy), scale));
  fx = fmin(fmax(fx, 0.0), qmax);
  fy = fmin(fmax(fy, 0.0), qmax);
  unsigned qx = (unsigned)fx, qy = (unsigned)fy;
  unsigned long long key = 0;
  for (int b = DEPTH_BITS - 1; b >= 0; b--)
    key = (key << 2) | ((unsigned long long)((qy >> b) & 1u) << 1) | (unsigned long long)((qx >> b) & 1u);
  keys[i] = key | ((unsigned long long)sidx << (2 * DEPTH_BITS));
  idx[i] = (int)i;
}

__global__ void gather_points_kernel(const double* __restrict__ pts, const int* __restrict__ perm,
                                     int64_t n, double* __restrict__ xt, int* __restrict__ iperm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = perm[i];
  xt[2 * i] = pts[2 * (int64_t)o];
  xt[2 * i + 1] = pts[2 * (int64_t)o + 1];
  iperm[o] = (int)i;
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (64-bit key, int index) pairs, 8-bit digits.  Per
// pass: per-tile digit counts (tile = RS_THREADS x RS_ROUNDS elements, in
// index order), an exclusive scan of the digit-major count table (digit d of
// tile b at d * ntiles + b), and a scatter in which every element's place is
// its tile's start for its digit plus its rank among the tile's earlier
// elements with the same digit (rounds of RS_THREADS consecutive elements;
// within a round, warps in order and lanes in order).
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) radix_count_kernel(const unsigned long long* __restrict__ keys,
                                                                 int64_t n, int shift, int ntiles,
                                                                 unsigned int* __restrict__ counts) {
  __shared__ unsigned int h[256];
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    const int64_t i = base + (int64_t)r * RS_THREADS + t;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)t * ntiles + blockIdx.x] = h[t];
}

// Exclusive scan of m counts in place, one CTA of 1024 threads (each scans a
// contiguous chunk, then the chunk totals are scanned).
__global__ void __launch_bounds__(1024) radix_scan_kernel(unsigned int* __restrict__ c, int64_t m) {
  __shared__ unsigned int part[1024];
  const int t = threadIdx.x;
  const int64_t per = (m + 1023) / 1024;
  const int64_t b = (int64_t)t * per, e = b + per < m ? b + per : m;
  unsigned int sum = 0;
  for (int64_t i = b; i < e; i++) sum += c[i];
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive Hillis-Steele scan of the chunk totals
    unsigned int v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned int run = t > 0 ? part[t - 1] : 0u;
  for (int64_t i = b; i < e; i++) {
    const unsigned int v = c[i];
    c[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(RS_THREADS) radix_scatter_kernel(
    const unsigned long long* __restrict__ kin, const int* __restrict__ vin, int64_t n, int shift, int ntiles,
    const unsigned int* __restrict__ offs, unsigned long long* __restrict__ kout, int* __restrict__ vout) {
  __shared__ unsigned int run[256];              // elements of each digit placed by earlier rounds
  __shared__ unsigned int wcnt[RS_WARPS][256];   // this pass of RS_THREADS elements: per warp and digit counts, then offsets
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  run[t] = offs[(int64_t)t * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; r++) {
    for (int k = 0; k < RS_WARPS; k++) wcnt[k][t] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)r * RS_THREADS + t;
    const bool valid = i < n;
    unsigned long long key = 0ull;
    int val = 0;
    unsigned d = 256u;   // no digit for elements past the end
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (unsigned)(key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {   // thread t owns digit t: offsets of the warps within the round
      unsigned acc = run[t];
      for (int k = 0; k < RS_WARPS; k++) {
        const unsigned c = wcnt[k][t];
        wcnt[k][t] = acc;
        acc += c;
      }
      run[t] = acc;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = wcnt[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

// Sorts (keys, vals) by the low end_bit bits of the keys; the result ends in
// (keys, vals) (ping-pong through the two scratch arrays).
static void radix_sort_pairs(DBuf& keys, DBuf& vals, DBuf& keys2, DBuf& vals2, int64_t n, int end_bit,
                             cudaStream_t s) {
  const int ntiles = (int)cdiv(n, RS_TILE);
  DBuf counts;
  counts.alloc(sizeof(unsigned int) * 256 * (int64_t)ntiles, s);
  for (int shift = 0; shift < end_bit; shift += 8) {
    LAUNCH(radix_count_kernel, ntiles, RS_THREADS, 0, s, keys.as<unsigned long long>(), n, shift, ntiles,
           counts.as<unsigned int>());
    LAUNCH(radix_scan_kernel, 1, 1024, 0, s, counts.as<unsigned int>(), (int64_t)256 * ntiles);
    LAUNCH(radix_scatter_kernel, ntiles, RS_THREADS, 0, s, keys.as<unsigned long long>(), vals.as<int>(), n, shift,
           ntiles, counts.as<unsigned int>(), keys2.as<unsigned long long>(), vals2.as<int>());
    std::swap(keys, keys2);
    std::swap(vals, vals2);
  }
}

// ------------------------------------------------------------- box table
// Breadth-first quadtree over the sorted keys, by one CTA: the roots of all
// sets first, then level by level the children (slots in Morton order) of
// every box of the previous level that holds more than n_occ points (and is
// above the deepest level); a child is the run of positions whose 2-bit digit
// at that level equals its slot, found by binary search in its parent's
// range.  Boxes get consecutive ids in that order.  Output per box: level,
// start, count, parent, slot, ix, iy, set; *nbox_out the number of boxes, or
// -1 when cap was too small.
struct BoxRow {
  int level, start, count, parent, slot, ix, iy, set;
};

__global__ void __launch_bounds__(1024) box_table_kernel(const unsigned long long* __restrict__ keys,
                                                         const int64_t* __restrict__ set_off, int nsets, int n_occ,
                                                         int cap, BoxRow* __restrict__ box, int* __restrict__ nbox_out) {
  __shared__ int s_run, s_tot[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (nsets > cap) {
    if (t == 0) *nbox_out = -1;
    return;
  }
  for (int i = t; i < nsets; i += 1024)
    box[i] = BoxRow{0, (int)set_off[i], (int)(set_off[i + 1] - set_off[i]), -1, 0, 0, 0, i};
  __syncthreads();
  int f0 = 0, f1 = nsets;   // the previous level's boxes
  int nb = nsets;
  for (int lev = 0; lev < DEPTH_BITS && f1 > f0; lev++) {
    const int shift = 2 * (DEPTH_BITS - lev - 1);
    if (t == 0) s_run = 0;
    __syncthreads();
    for (int c0 = f0; c0 < f1; c0 += 1024) {   // chunks of parents, in order
      const int b = c0 + t;
      int bounds[5] = {0, 0, 0, 0, 0};
      int made = 0;
      BoxRow P{};
      if (b < f1) {
        P = box[b];
        if (P.count > n_occ) {
          for (int sl = 0; sl <= 4; sl++) {
            int lo = P.start, hi = P.start + P.count;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if ((int)((keys[mid] >> shift) & 3ull) < sl) lo = mid + 1;
              else hi = mid;
            }
            bounds[sl] = lo;
          }
          for (int sl = 0; sl < 4; sl++) made += bounds[sl + 1] > bounds[sl];
        }
      }
      // exclusive scan of "made" over the chunk (warp shuffles, then warps)
      int inc = made;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
      }
      if (lane == 31) s_tot[w] = inc;
      __syncthreads();
      if (w == 0) {
        int v = s_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        s_tot[lane] = v;   // inclusive over warps
      }
      __syncthreads();
      const int before = (w > 0 ? s_tot[w - 1] : 0) + inc - made;
      const int id0 = nb + s_run + before;
      if (made > 0 && id0 + made <= cap) {
        int k = 0;
        for (int sl = 0; sl < 4; sl++)
          if (bounds[sl + 1] > bounds[sl])
            box[id0 + k++] = BoxRow{lev + 1, bounds[sl], bounds[sl + 1] - bounds[sl], b, sl,
                                    2 * P.ix + (sl & 1), 2 * P.iy + (sl >> 1), P.set};
      }
      __syncthreads();
      if (t == 0) s_run += s_tot[31];
      __syncthreads();
    }
    f0 = nb;
    nb += s_run;
    f1 = nb;
    if (nb > cap) break;
    __syncthreads();
  }
  if (t == 0) *nbox_out = nb > cap ? -1 : nb;
}

// Index of every tree position within its leaf.
__global__ void leafpos_kernel(const BoxRow* __restrict__ box, const char* __restrict__ leaf, int nbox,
                               int* __restrict__ leafpos) {
  const int b = blockIdx.x;
  if (b >= nbox || !leaf[b]) return;
  const BoxRow B = box[b];
  for (int i = threadIdx.x; i < B.count; i += blockDim.x) leafpos[B.start + i] = i;
}

std::shared_ptr<rsf_tree_s> build_forest(const double* points, const std::vector<int64_t>& set_off,
                                         const rsf_opts& o, cudaStream_t s) {
  const int nsets = (int)set_off.size() - 1;
  RSF_CHECK(nsets >= 1 && nsets <= (1 << 14), RSF_EINVAL, "number of point sets out of range (1 .. 16384)");
  RSF_CHECK(set_off[0] == 0, RSF_EINVAL, "set offsets must start at 0");
  for (int i = 0; i < nsets; i++)
    RSF_CHECK(set_off[i + 1] > set_off[i], RSF_EINVAL, "every point set must hold at least one point");
  const int64_t n = set_off[nsets];
  RSF_CHECK(n > 0 && n < (int64_t)1 << 31, RSF_EINVAL, "n out of range");
  RSF_CHECK(o.n_occ >= 1, RSF_EINVAL, "n_occ must be >= 1");
  auto tr = std::make_shared<rsf_tree_s>();
  tr->opts = o;
  TreeData& T = tr->t;
  T.n = n;
  T.n_occ = o.n_occ;
  T.stream = s;
  T.nsets = nsets;
  T.set_off = set_off;
  // bounding box of every set
  std::vector<int> nblk(nsets), blk0(nsets + 1, 0);
  for (int i = 0; i < nsets; i++) {
    nblk[i] = (int)std::min<int64_t>(1024, std::max<int64_t>(1, cdiv(set_off[i + 1] - set_off[i], 256)));
    blk0[i + 1] = blk0[i] + nblk[i];
  }
  DBuf part;
  part.alloc(sizeof(double) * 4 * blk0[nsets], s);
  for (int i = 0; i < nsets; i++)
    LAUNCH(bbox_partial_kernel, nblk[i], 256, 0, s, points + 2 * set_off[i], set_off[i + 1] - set_off[i],
           part.as<double>() + 4 * blk0[i]);
  std::vector<double> hp(4 * blk0[nsets]);
  d2h(hp.data(), part.as<double>(), hp.size(), s);
  sync(s);
  T.set_lo.assign(2 * nsets, 0.0);
  T.set_side.assign(nsets, 1.0);
  std::vector<double> geom(3 * nsets);
  for (int i = 0; i < nsets; i++) {
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int b = blk0[i]; b < blk0[i + 1]; b++) {
      xmin = std::min(xmin, hp[4 * b]); xmax = std::max(xmax, hp[4 * b + 1]);
      ymin = std::min(ymin, hp[4 * b + 2]); ymax = std::max(ymax, hp[4 * b + 3]);
    }
    RSF_CHECK(std::isfinite(xmin) && std::isfinite(xmax) && std::isfinite(ymin) && std::isfinite(ymax),
              RSF_EINVAL, "points contain NaN or Inf");
    double side = std::max(xmax - xmin, ymax - ymin);
    if (!(side > 0.0)) side = 1.0;
    volatile double half = 0.5;  // keep the host arithmetic identical to the oracle's
    double cx = (xmin + xmax) * half, cy = (ymin + ymax) * half;
    T.set_side[i] = side;
    T.set_lo[2 * i] = cx - side * half;
    T.set_lo[2 * i + 1] = cy - side * half;
    geom[3 * i] = T.set_lo[2 * i];
    geom[3 * i + 1] = T.set_lo[2 * i + 1];
    geom[3 * i + 2] = (double)(1u << DEPTH_BITS) / side;
  }
  T.side = T.set_side[0];
  T.lo[0] = T.set_lo[0];
  T.lo[1] = T.set_lo[1];
  // keys + sort (the set index above the Morton bits)
  int set_bits = 0;
  while ((1 << set_bits) < nsets) set_bits++;
  DBuf keys, keys2, idx, idx2, bad, doff, dgeom;
  upload(doff, set_off, s);
  upload(dgeom, geom, s);
  keys.alloc(sizeof(unsigned long long) * n, s);
  keys2.alloc(sizeof(unsigned long long) * n, s);
  idx.alloc(sizeof(int) * n, s);
  idx2.alloc(sizeof(int) * n, s);
  bad.alloc(sizeof(int), s);
  bad.zero();
  LAUNCH(keys_kernel, cdiv(n, 256), 256, 0, s, points, n, doff.as<int64_t>(), nsets, dgeom.as<double>(),
         keys.as<unsigned long long>(), idx.as<int>(), bad.as<int>());
  radix_sort_pairs(keys, idx, keys2, idx2, n, 2 * DEPTH_BITS + set_bits, s);
  int hbad = 0;
  d2h(&hbad, bad.as<int>(), 1, s);
  // tree-order coordinates
  T.perm = std::move(idx);
  T.xt.alloc(sizeof(double) * 2 * n, s);
  T.iperm.alloc(sizeof(int) * n, s);
  LAUNCH(gather_points_kernel, cdiv(n, 256), 256, 0, s, points, T.perm.as<int>(), n,
         T.xt.as<double>(), T.iperm.as<int>());
  sync(s);
  RSF_CHECK(!hbad, RSF_EINVAL, "points contain NaN or Inf");

  // box table on the device; the capacity starts near the usual count
  // (about n / n_occ boxes per level of splitting) and grows on overflow
  std::vector<BoxRow> rows;
  {
    int64_t cap = nsets + 8 * (n / (o.n_occ + 1) + 1) + 1024;
    const int64_t cap_max = nsets + 4 * (int64_t)DEPTH_BITS * (n / (o.n_occ + 1) + 1);
    DBuf dbox, dnb;
    dnb.alloc(sizeof(int), s);
    for (;;) {
      const int64_t c = std::min(cap, cap_max);
      RSF_CHECK(c < (int64_t)1 << 31, RSF_EINVAL, "too many boxes");
      dbox.alloc(sizeof(BoxRow) * c, s);
      LAUNCH(box_table_kernel, 1, 1024, 0, s, keys.as<unsigned long long>(), doff.as<int64_t>(), nsets, o.n_occ,
             (int)c, dbox.as<BoxRow>(), dnb.as<int>());
      int nbh = 0;
      d2h(&nbh, dnb.as<int>(), 1, s);
      sync(s);
      if (nbh >= 0) {
        rows.resize(nbh);
        d2h(rows.data(), dbox.as<BoxRow>(), nbh, s);
        sync(s);
        break;
      }
      RSF_CHECK(c < cap_max, RSF_ECUDA, "box table: capacity bound exceeded");
      cap *= 4;
    }
    const int nbox = (int)rows.size();
    T.level.resize(nbox); T.start.resize(nbox); T.count.resize(nbox); T.parent.resize(nbox);
    T.slot.resize(nbox); T.ix.resize(nbox); T.iy.resize(nbox); T.box_set.resize(nbox);
    T.children.assign(nbox, {-1, -1, -1, -1});
    for (int b = 0; b < nbox; b++) {
      const BoxRow& r = rows[b];
      T.level[b] = r.level; T.start[b] = r.start; T.count[b] = r.count; T.parent[b] = r.parent;
      T.slot[b] = r.slot; T.ix[b] = r.ix; T.iy[b] = r.iy; T.box_set[b] = r.set;
      if (r.parent >= 0) T.children[r.parent][r.slot] = b;
    }
    // per-position index within its leaf, on the device
    std::vector<char> leaf(nbox);
    for (int b = 0; b < nbox; b++)
      leaf[b] = T.children[b][0] < 0 && T.children[b][1] < 0 && T.children[b][2] < 0 && T.children[b][3] < 0;
    DBuf dleaf;
    upload(dleaf, leaf, s);
    T.leafpos_d.alloc(sizeof(int) * n, s);
    LAUNCH(leafpos_kernel, nbox, 128, 0, s, dbox.as<BoxRow>(), dleaf.as<char>(), nbox, T.leafpos_d.as<int>());
  }
  int nbox = (int)T.level.size();
  T.is_leaf.resize(nbox);
  T.cx.resize(nbox); T.cy.resize(nbox); T.w.resize(nbox);
  T.L = 0;
  for (int b = 0; b < nbox; b++) {
    T.is_leaf[b] = T.children[b][0] < 0 && T.children[b][1] < 0 && T.children[b][2] < 0 && T.children[b][3] < 0;
    T.L = std::max(T.L, T.level[b]);
    const int si = T.box_set[b];
    double w = T.set_side[si] / std::ldexp(1.0, T.level[b]);
    T.w[b] = w;
    T.cx[b] = T.set_lo[2 * si] + (T.ix[b] + 0.5) * w;
    T.cy[b] = T.set_lo[2 * si + 1] + (T.iy[b] + 0.5) * w;
    if (T.is_leaf[b]) T.max_leaf = std::max(T.max_leaf, T.count[b]);
  }
  T.by_level.assign(T.L + 1, {});
  for (int b = 0; b < nbox; b++) T.by_level[T.level[b]].push_back(b);
  upload(T.box_set_d, T.box_set, s);
  upload(T.set_off_d, T.set_off, s);
  return tr;
}

std::shared_ptr<rsf_tree_s> build_tree(const double* points, int64_t n, const rsf_opts& o, cudaStream_t s) {
  RSF_CHECK(n > 0 && n < (int64_t)1 << 31, RSF_EINVAL, "n out of range");
  return build_forest(points, std::vector<int64_t>{0, n}, o, s);
}

}  // namespace rsf
