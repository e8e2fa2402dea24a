// Quadtree construction (Sec. 2.1, Remark (tree)).
//
// Device: bounding box reduction, quantised coordinates and Morton keys
// (D = 24 bits per axis, y bit above x bit, so child slots are SW, SE, NW,
// NE), a stable radix sort of (key, index) -- ties keep the original index
// order -- and the gather of the coordinates into tree order.  Host: the box
// table (split while a box holds more than n_occ points), derived from the
// sorted keys with binary searches; it is small (O(n / n_occ) boxes) and the
// host needs it to size every level.
//
// A forest of independent point sets (batched datasets) is built the same
// way: every set gets its own root square, its set index sits above the 48
// Morton bits of the key, so one radix sort groups the sets (in order) and
// orders each set's points; every box records its set.  Boxes of different
// sets never interact.
#include <cub/device/device_radix_sort.cuh>

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
  size_t tmp_bytes = 0;
  const int end_bit = 2 * DEPTH_BITS + set_bits;
  RSF_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys.as<unsigned long long>(),
                                           keys2.as<unsigned long long>(), idx.as<int>(), idx2.as<int>(),
                                           (int)n, 0, end_bit, s));
  DBuf tmp;
  tmp.alloc(std::max<size_t>(tmp_bytes, 16), s);
  RSF_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, keys.as<unsigned long long>(),
                                           keys2.as<unsigned long long>(), idx.as<int>(), idx2.as<int>(),
                                           (int)n, 0, end_bit, s));
  g_launches += 4;  // the radix sort's own passes (approximate count)
  std::vector<unsigned long long> hk(n);
  d2h(hk.data(), keys2.as<unsigned long long>(), n, s);
  int hbad = 0;
  d2h(&hbad, bad.as<int>(), 1, s);
  // tree-order coordinates
  T.perm = std::move(idx2);
  T.xt.alloc(sizeof(double) * 2 * n, s);
  T.iperm.alloc(sizeof(int) * n, s);
  LAUNCH(gather_points_kernel, cdiv(n, 256), 256, 0, s, points, T.perm.as<int>(), n,
         T.xt.as<double>(), T.iperm.as<int>());
  sync(s);
  RSF_CHECK(!hbad, RSF_EINVAL, "points contain NaN or Inf");

  // Box table, breadth first (same rule as the quadtree description above);
  // the roots of all sets first, so the levels stay contiguous.
  auto add_box = [&](int lev, int st, int ct, int par, int sl, int bx, int by, int set) {
    T.level.push_back(lev); T.start.push_back(st); T.count.push_back(ct);
    T.parent.push_back(par); T.slot.push_back(sl); T.ix.push_back(bx); T.iy.push_back(by);
    T.box_set.push_back(set);
    T.children.push_back({-1, -1, -1, -1});
    return (int)T.level.size() - 1;
  };
  std::vector<int> frontier;
  for (int i = 0; i < nsets; i++)
    frontier.push_back(add_box(0, (int)set_off[i], (int)(set_off[i + 1] - set_off[i]), -1, 0, 0, 0, i));
  int lev = 0;
  while (!frontier.empty()) {
    std::vector<int> next;
    for (int b : frontier) {
      if (T.count[b] <= o.n_occ || lev >= DEPTH_BITS) continue;
      int s0 = T.start[b], c0 = T.count[b];
      int shift = 2 * (DEPTH_BITS - lev - 1);
      int bounds[5];
      for (int sl = 0; sl <= 4; sl++) {
        // first position in [s0, s0+c0) whose 2-bit digit at this level >= sl
        int lo = s0, hi = s0 + c0;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if ((int)((hk[mid] >> shift) & 3ull) < sl) lo = mid + 1; else hi = mid;
        }
        bounds[sl] = lo;
      }
      for (int sl = 0; sl < 4; sl++) {
        if (bounds[sl + 1] > bounds[sl]) {
          int c = add_box(lev + 1, bounds[sl], bounds[sl + 1] - bounds[sl], b, sl,
                          2 * T.ix[b] + (sl & 1), 2 * T.iy[b] + (sl >> 1), T.box_set[b]);
          T.children[b][sl] = c;
          next.push_back(c);
        }
      }
    }
    frontier.swap(next);
    lev++;
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
  T.leafpos.assign(n, 0);
  for (int b = 0; b < nbox; b++)
    if (T.is_leaf[b])
      for (int i = 0; i < T.count[b]; i++) T.leafpos[T.start[b] + i] = i;
  upload(T.box_set_d, T.box_set, s);
  upload(T.set_off_d, T.set_off, s);
  return tr;
}

std::shared_ptr<rsf_tree_s> build_tree(const double* points, int64_t n, const rsf_opts& o, cudaStream_t s) {
  RSF_CHECK(n > 0 && n < (int64_t)1 << 31, RSF_EINVAL, "n out of range");
  return build_forest(points, std::vector<int64_t>{0, n}, o, s);
}

}  // namespace rsf
