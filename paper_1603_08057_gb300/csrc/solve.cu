// Multi-right-hand-side application of the factorization (Sec. 2.3.2):
// F = Q D Q^T with Q = prod_l prod_I L_I U_I (leaf level leftmost) and D the
// block-diagonal of the X_RR blocks and the root block.
//
//   Q^-1 (leaves first):   x_R -= T^T x_S ;  x_S -= E x_R
//   Q^-T (root side first): x_R -= E^T x_S ;  x_S -= T x_R
//   Q^T  (leaves first):   x_S += T x_R   ;  x_R += E^T x_S
//   Q    (root side first): x_S += E x_R   ;  x_R += T^T x_S
//   F^-1 = Q^-T D^-1 Q^-1, F = Q D Q^T, F^1/2 = Q C, F^-1/2 = C^-1 Q^-1.
//
// Work buffers: one row-major (rows x q) block per level holding the active
// DOFs of that level in [S, R] order per box; the skeleton rows move between
// levels through the gather map built with the factorization.  Every box
// operation of a level is one batched GEMM launch.
#include <algorithm>

#include "df64.cuh"
#include "internal.cuh"

namespace rsf {

// X_lev[row] = src >= 0 ? X_up[src] : in[-(1 + src)]   (row length q); rows
// taken from the input are converted to df64 pairs when cvt is set.
__global__ void gather_rows_kernel(const int* __restrict__ src, int64_t nrows, int q,
                                   const double* __restrict__ child, const double* __restrict__ in,
                                   double* __restrict__ out, int cvt) {
  int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int s = src[row];
  const double* from = s >= 0 ? child + (int64_t)s * q : in + (int64_t)(-(1 + s)) * q;
  double* to = out + row * q;
  if (cvt && s < 0) {
    for (int c = lane; c < q; c += 32) {
      df64 v = df_from_double(from[c]);
      reinterpret_cast<float2*>(to)[c] = make_float2(v.hi, v.lo);
    }
  } else {
    for (int c = lane; c < q; c += 32) to[c] = from[c];
  }
}

// Inverse of the gather: rows with src >= 0 go back to the level below, leaf
// rows to the output.
__global__ void scatter_rows_kernel(const int* __restrict__ src, int64_t nrows, int q,
                                    const double* __restrict__ lev, double* __restrict__ child,
                                    double* __restrict__ out, int cvt) {
  int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  int s = src[row];
  double* to = s >= 0 ? child + (int64_t)s * q : out + (int64_t)(-(1 + s)) * q;
  const double* from = lev + row * q;
  if (cvt && s < 0) {
    for (int c = lane; c < q; c += 32) {
      float2 f = reinterpret_cast<const float2*>(from)[c];
      to[c] = df_to_double({f.x, f.y});
    }
  } else {
    for (int c = lane; c < q; c += 32) to[c] = from[c];
  }
}

__global__ void convert_df64_kernel(double* __restrict__ p, int64_t n, int to) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  if (to) {
    df64 v = df_from_double(p[g]);
    reinterpret_cast<float2*>(p)[g] = make_float2(v.hi, v.lo);
  } else {
    float2 f = reinterpret_cast<const float2*>(p)[g];
    p[g] = df_to_double({f.x, f.y});
  }
}

void convert_df64(double* p, int64_t n, int to, cudaStream_t s) {
  if (n > 0) LAUNCH(convert_df64_kernel, cdiv(n, 256), 256, 0, s, p, n, to);
}

// Copy the R rows (ranges) of a level between two buffers.
__global__ void copy_ranges_kernel(const int64_t* __restrict__ rr, int nrr, int q,
                                   const double* __restrict__ from, double* __restrict__ to) {
  int i = blockIdx.x;
  if (i >= nrr) return;
  int64_t r0 = rr[2 * i], nr = rr[2 * i + 1];
  const double* f = from + r0 * q;
  double* t = to + r0 * q;
  for (int64_t e = threadIdx.x; e < nr * q; e += blockDim.x) t[e] = f[e];
}

static void run_level_gemm(const GemmBatch& g, double* X, double* tmp, double* pool, int q, double alpha,
                           cudaStream_t s, int df) {
  GemmBases b{};
  b.df = df;
  b.p[0] = X; b.p[1] = tmp; b.p[2] = pool; b.p[3] = nullptr;
  b.sc[0] = q; b.sc[1] = q; b.sc[2] = 1; b.sc[3] = 1;
  b.M = q; b.ld = q; b.alpha_scale = alpha;
  g.run(b, s);
}

// The descriptors of one level restricted to each box's nonzero column block.
static void restrict_batch(const std::vector<GemmDesc>& d, const std::vector<int>& box, const std::vector<int>& slot,
                           int qc, cudaStream_t s, GemmBatch& out) {
  std::vector<GemmDesc> r;
  r.reserve(d.size());
  for (size_t j = 0; j < d.size(); j++) {
    const int sl = slot[box[j]];
    if (sl < 0) continue;
    GemmDesc g = d[j];
    g.M = qc;
    g.m0 = sl * qc;
    r.push_back(g);
  }
  out.build(r, s);
}

// The descriptors of one level without each box's unneeded column block
// (boxes without a slot keep all columns).
static void complement_batch(const std::vector<GemmDesc>& d, const std::vector<int>& box,
                             const std::vector<int>& slot, int qc, int nblk, cudaStream_t s, GemmBatch& out) {
  std::vector<GemmDesc> r;
  r.reserve(2 * d.size());
  for (size_t j = 0; j < d.size(); j++) {
    const int sl = slot[box[j]];
    GemmDesc g = d[j];
    if (sl < 0) {
      g.M = nblk * qc;
      g.m0 = 0;
      r.push_back(g);
      continue;
    }
    if (sl > 0) {
      g.M = sl * qc;
      g.m0 = 0;
      r.push_back(g);
    }
    if (sl < nblk - 1) {
      g.M = (nblk - 1 - sl) * qc;
      g.m0 = (sl + 1) * qc;
      r.push_back(g);
    }
  }
  out.build(r, s);
}

void solve_rows(rsf_handle_s* h, int op, const double* in, double* out, int q, int io_df, const SparseRHS* sp,
                const SparseRHS* skip_out) {
  RSF_CHECK(!skip_out || (skip_out->qc > 0 && q % skip_out->qc == 0), RSF_EINVAL, "column blocks must tile q");
  const int nblk = skip_out ? q / skip_out->qc : 1;
  const int df = h->df;
  const int cvt = (df && !io_df) ? 1 : 0;
  RSF_CHECK(!io_df || df, RSF_EINVAL, "df64 input needs a mixed-precision factorization");
  cudaStream_t s = h->stream;
  const int L = (int)h->levels.size() - 1;
  RSF_CHECK(q >= 1, RSF_EINVAL, "nrhs must be >= 1");
  if (!h->spd) RSF_CHECK(op == RSF_OP_APPLY, RSF_EINVAL, "only APPLY is defined for a derivative factorization");
  // buffers
  std::vector<int64_t> off(L + 2, 0);
  int64_t maxrows = 0;
  for (int l = 0; l <= L; l++) {
    off[l + 1] = off[l] + h->levels[l].nrows;
    maxrows = std::max(maxrows, h->levels[l].nrows);
  }
  DBuf X, tmp;
  X.alloc(sizeof(double) * std::max<int64_t>(1, off[L + 1]) * q, s);
  tmp.alloc(sizeof(double) * std::max<int64_t>(1, maxrows) * q, s);
  auto Xl = [&](int l) { return X.as<double>() + off[l] * q; };

  int up = 0, down = 0, mid = 0;  // up/down: 0 none, 1 inverse, 2 forward
  switch (op) {
    case RSF_OP_INV: up = 1; down = 1; mid = 0; break;
    case RSF_OP_APPLY: up = 2; down = 2; mid = 1; break;
    case RSF_OP_SQRT: up = 0; down = 2; mid = 2; break;
    case RSF_OP_SQRT_T: up = 2; down = 0; mid = 3; break;
    case RSF_OP_INV_SQRT: up = 1; down = 0; mid = 4; break;
    case RSF_OP_INV_SQRT_T: up = 0; down = 1; mid = 5; break;
    default: fail(RSF_EINVAL, "unknown op");
  }
  // upward sweep
  for (int l = L; l >= 0; l--) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrows == 0) continue;
    const double* child = (l < L) ? Xl(l + 1) : nullptr;
    LAUNCH(gather_rows_kernel, cdiv(Lv.nrows, 8), 256, 0, s, Lv.src.as<int>(), Lv.nrows, q, child, in, Xl(l), cvt);
    if (l == 0) break;
    double* F = Lv.fpool.as<double>();
    const bool sparse = sp && l >= sp->lev0;
    GemmBatch r1, r2;
    if (up == 1) {
      const GemmBatch* g1 = &Lv.gRS_T;
      const GemmBatch* g2 = &Lv.gSR_Et;
      if (sparse) {
        restrict_batch(Lv.hRS_T, Lv.boxRSE, sp->slot[l], sp->qc, s, r1);
        restrict_batch(Lv.hSR_Et, Lv.boxRSE, sp->slot[l], sp->qc, s, r2);
        g1 = &r1; g2 = &r2;
      }
      run_level_gemm(*g1, Xl(l), tmp.as<double>(), F, q, -1.0, s, df);
      run_level_gemm(*g2, Xl(l), tmp.as<double>(), F, q, -1.0, s, df);
    } else if (up == 2) {
      const GemmBatch* g1 = &Lv.gSR_Tt;
      const GemmBatch* g2 = &Lv.gRS_E;
      if (sparse) {
        restrict_batch(Lv.hSR_Tt, Lv.boxRSE, sp->slot[l], sp->qc, s, r1);
        restrict_batch(Lv.hRS_E, Lv.boxRSE, sp->slot[l], sp->qc, s, r2);
        g1 = &r1; g2 = &r2;
      }
      run_level_gemm(*g1, Xl(l), tmp.as<double>(), F, q, 1.0, s, df);
      run_level_gemm(*g2, Xl(l), tmp.as<double>(), F, q, 1.0, s, df);
    }
  }
  // block-diagonal middle factor on the R rows of every level
  for (int l = 0; l <= L; l++) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrr == 0) continue;
    double* F = Lv.fpool.as<double>();
    double* x = Xl(l);
    double* t = tmp.as<double>();
    const bool sparse = sp && l >= sp->lev0;
    const bool skip = skip_out && l >= skip_out->lev0;
    auto prod = [&](int v, bool from_tmp) {
      // out = in * op(B): descriptors read base 0 and write base 1; on a
      // sparse level only each box's nonzero column block (the others stay
      // zero in x)
      GemmBases b{};
      b.p[0] = from_tmp ? t : x; b.p[1] = from_tmp ? x : t; b.p[2] = F; b.p[3] = nullptr;
      b.sc[0] = q; b.sc[1] = q; b.sc[2] = 1; b.sc[3] = 1;
      b.M = q; b.ld = q; b.alpha_scale = 1.0;
      b.df = df;
      if (sparse) {
        GemmBatch r;
        restrict_batch(Lv.hMid[v], Lv.boxMid[v], sp->slot[l], sp->qc, s, r);
        r.run(b, s);
      } else if (skip) {
        GemmBatch r;
        complement_batch(Lv.hMid[v], Lv.boxMid[v], skip_out->slot[l], skip_out->qc, nblk, s, r);
        r.run(b, s);
      } else {
        Lv.gMid[v].run(b, s);
      }
    };
    auto copy_to_tmp = [&]() {
      LAUNCH(copy_ranges_kernel, Lv.nrr, 256, 0, s, Lv.rr.as<int64_t>(), Lv.nrr, q, x, t);
    };
    switch (mid) {
      case 0: prod(0, false); prod(1, true); break;             // D^-1 = Cinv^T Cinv
      case 1:
        if (h->spd) { prod(2, false); prod(3, true); }           // D = C C^T
        else { copy_to_tmp(); prod(4, true); }                   // D = X_RR
        break;
      case 2: copy_to_tmp(); prod(3, true); break;               // C
      case 3: copy_to_tmp(); prod(2, true); break;               // C^T
      case 4: copy_to_tmp(); prod(0, true); break;               // C^-1
      case 5: copy_to_tmp(); prod(1, true); break;               // C^-T
    }
  }
  // downward sweep
  for (int l = 0; l <= L; l++) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrows == 0) continue;
    double* F = Lv.fpool.as<double>();
    if (l > 0 && down != 0) {
      const bool skip = skip_out && l >= skip_out->lev0;
      const GemmBatch* g1 = down == 1 ? &Lv.gRS_E : &Lv.gSR_Et;
      const GemmBatch* g2 = down == 1 ? &Lv.gSR_Tt : &Lv.gRS_T;
      GemmBatch r1, r2;
      if (skip) {
        complement_batch(down == 1 ? Lv.hRS_E : Lv.hSR_Et, Lv.boxRSE, skip_out->slot[l], skip_out->qc, nblk, s, r1);
        complement_batch(down == 1 ? Lv.hSR_Tt : Lv.hRS_T, Lv.boxRSE, skip_out->slot[l], skip_out->qc, nblk, s, r2);
        g1 = &r1; g2 = &r2;
      }
      const double a = down == 1 ? -1.0 : 1.0;
      run_level_gemm(*g1, Xl(l), tmp.as<double>(), F, q, a, s, df);
      run_level_gemm(*g2, Xl(l), tmp.as<double>(), F, q, a, s, df);
    }
    double* child = (l < L) ? Xl(l + 1) : nullptr;
    LAUNCH(scatter_rows_kernel, cdiv(Lv.nrows, 8), 256, 0, s, Lv.src.as<int>(), Lv.nrows, q, Xl(l), child, out, cvt);
  }
}

// ------------------------------------------------------------- reductions
__global__ void dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                   double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
    s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

void dot_into(const double* a, const double* b, int64_t n, double* d_out, cudaStream_t s) {
  int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, cdiv(n, 256)));
  DBuf part;
  part.alloc(sizeof(double) * nb, s);
  LAUNCH(dot_partial_kernel, nb, 256, 0, s, a, b, n, part.as<double>());
  LAUNCH(sum_kernel, 1, 256, 0, s, part.as<double>(), nb, d_out);
}

double dot_device(const double* a, const double* b, int64_t n, cudaStream_t s) {
  int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, cdiv(n, 256)));
  DBuf part, res;
  part.alloc(sizeof(double) * nb, s);
  res.alloc(sizeof(double), s);
  LAUNCH(dot_partial_kernel, nb, 256, 0, s, a, b, n, part.as<double>());
  LAUNCH(sum_kernel, 1, 256, 0, s, part.as<double>(), nb, res.as<double>());
  double h = 0;
  d2h(&h, res.as<double>(), 1, s);
  sync(s);
  return h;
}

}  // namespace rsf
