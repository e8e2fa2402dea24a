// Trace of a symmetric black-box operator by weak-admissibility peeling
// (Sec. 3), G = F^-1 or G = (F^-1 F_k + F_k F^-1)/2 (Algorithm 1).
//
// Level l = 1..L, top down:
//   * test matrices W_k (k = slot 0..3) with i.i.d. N(0,1) entries on the rows
//     of the level-l boxes in child slot k, zero elsewhere (Sec. 3.2); drawn
//     from Philox4x32-10 with counter (row, col/4, level, 0), Box-Muller;
//   * Y_k = G W_k - sum_{m<l} G^(m) W_k (all four slots in one multi-RHS
//     application);
//   * every ordered sibling pair (a, b): Y_ab = Y_{slot(b)}(I_a, :) ~ G_ab W_b;
//     column-pivoted QR with relative cut-off tol gives the rank r_ab and the
//     basis U_ab = Y_ab(:, piv) R11^-1;
//   * Eq. (lowrankapprox): M_ab = (W_a^T U_ab)^+ Z (U_ba^T W_b)^+ with the
//     symmetrised core Z = (W_a^T Y_ab + (W_b^T Y_ba)^T)/2 and M_ba = M_ab^T;
//   * adaptivity: if a rank exceeds q - c, another q columns are appended.
// Finally H = (G - sum_m G^(m)) E with E the stacked leaf identities and
// Tr(G) ~ sum_leaves Tr H(I_i, [n_i]) (Sec. 3.2.4).
#include <algorithm>
#include <cmath>

#include "df64.cuh"
#include "internal.cuh"

namespace rsf {

// --------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    unsigned long long p0 = (unsigned long long)0xD2511F53u * c[0];
    unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c[2];
    unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
    unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
    unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__device__ __forceinline__ double philox_normal(unsigned row, unsigned col, unsigned level, unsigned stream,
                                                unsigned long long seed) {
  unsigned c[4] = {row, col >> 2, level, stream};
  philox4x32_10(c, (unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32));
  const double two32 = 4294967296.0;
  int w = col & 3;
  double ua = ((double)c[w < 2 ? 0 : 2] + 0.5) / two32;
  double ub = ((double)c[w < 2 ? 1 : 3] + 0.5) / two32;
  double rad = sqrt(-2.0 * log(ua));
  double s, co;
  sincospi(2.0 * ub, &s, &co);
  return (w & 1) ? rad * s : rad * co;
}

__device__ __forceinline__ void store_val(double* p, double v, int df) {
  if (df) {
    df64 d = df_from_double(v);
    *reinterpret_cast<float2*>(p) = make_float2(d.hi, d.lo);
  } else {
    *p = v;
  }
}
__device__ __forceinline__ double load_val(const double* p, int df) {
  if (df) {
    float2 f = *reinterpret_cast<const float2*>(p);
    return df_to_double({f.x, f.y});
  }
  return *p;
}

// W chunk: n x (4 qc) row-major; row p of a level box in slot s gets the
// normals of columns col0 .. col0+qc-1 in column block s.
__global__ void gen_w_kernel(const int* __restrict__ slotrow, int64_t n, int qc, int col0, int level,
                             unsigned long long seed, double* __restrict__ W, int df) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tot = n * 4 * qc;
  if (g >= tot) return;
  int64_t p = g / (4 * qc);
  int c = (int)(g % (4 * qc));
  int s = slotrow[p];
  double v = 0.0;
  if (s >= 0 && c / qc == s) v = philox_normal((unsigned)p, (unsigned)(col0 + c % qc), (unsigned)level, 0u, seed);
  store_val(W + g, v, df);
}

// Column block extraction from row-major chunks into column-major matrices:
// out[i + (col0 + j) * ldo] = in[(r0 + i) * ldi + cb + j], i < rows, j < qc.
struct ExtractProb {
  int64_t r0, out0;
  int rows, cb;
};
// Sparse sign embedding of a sample block: out (ell x q, column-major, ld
// ell) = Omega Y with Omega given per bucket (row of Omega) as a list of
// (row of Y << 1 | negative sign), scaled by 1 / sqrt(SKETCH_S).  One thread
// per output entry, buckets fastest.
constexpr int SKETCH_S = 8;
struct SketchProb {
  int64_t y0, out0;   // Y block (rows x q, column-major, ld rows) and output offsets
  int rows;
  int bucket0;        // first bucket pointer of the box's embedding
};
__global__ void sparse_sketch_kernel(const SketchProb* __restrict__ sp, int64_t total, int ell, int q,
                                     const int* __restrict__ bptr, const int* __restrict__ ent,
                                     const double* __restrict__ Y, double* __restrict__ out, int df) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int64_t per = (int64_t)ell * q;
  const SketchProb P = sp[g / per];
  const int64_t rem = g % per;
  const int c = (int)(rem / ell), u = (int)(rem % ell);
  const double* y = Y + P.y0 + (int64_t)c * P.rows;
  double acc = 0.0;
  for (int k = bptr[P.bucket0 + u]; k < bptr[P.bucket0 + u + 1]; k++) {
    const int e = ent[k];
    const double v = load_val(y + (e >> 1), df);
    acc += (e & 1) ? -v : v;
  }
  out[P.out0 + u + (int64_t)c * ell] = acc * 0.35355339059327373;   // 1 / sqrt(8)
}

__global__ void extract_kernel(const ExtractProb* __restrict__ ep, const int64_t* __restrict__ prefix, int nprob,
                               int64_t total, int qc, int ldi, int col0, const double* __restrict__ in,
                               double* __restrict__ out, int df) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const ExtractProb e = ep[lo];
  int64_t x = g - prefix[lo];
  int i = (int)(x % e.rows), j = (int)(x / e.rows);
  out[e.out0 + i + (int64_t)(col0 + j) * e.rows] = load_val(in + (e.r0 + i) * ldi + e.cb + j, df);
}

// Gather pivot columns: out[:, t] = Y[:, piv[t]] for t < k.
struct PivGather {
  int64_t y0, out0, col0;
  int rows, ldy;
};
__global__ void pivgather_kernel(const PivGather* __restrict__ pg, const int64_t* __restrict__ prefix, int nprob,
                                 int64_t total, const int* __restrict__ piv, const QRState* __restrict__ st,
                                 const double* __restrict__ Y, double* __restrict__ out) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const PivGather e = pg[lo];
  int64_t x = g - prefix[lo];
  int i = (int)(x % e.rows), t = (int)(x / e.rows);
  if (t >= st[lo].k) return;
  int c = piv[e.col0 + t];
  out[e.out0 + i + (int64_t)t * e.rows] = Y[e.y0 + i + (int64_t)c * e.ldy];
}

// Least-squares scatter: out[o0 + piv[i]*ri + s*rs] = t[t0 + i + s*kq].
struct PermScatter {
  int64_t t0, o0, col0;
  int nrow, ncol, ri, rs;
};
__global__ void permscatter_kernel(const PermScatter* __restrict__ ps, const int64_t* __restrict__ prefix,
                                   int nprob, int64_t total, const int* __restrict__ piv,
                                   const QRState* __restrict__ st, const double* __restrict__ t,
                                   double* __restrict__ out) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const PermScatter e = ps[lo];
  int64_t x = g - prefix[lo];
  int i = (int)(x % e.nrow), s = (int)(x / e.nrow);
  int kq = st[lo].k;
  if (i >= kq) return;
  out[e.o0 + (int64_t)piv[e.col0 + i] * e.ri + (int64_t)s * e.rs] = t[e.t0 + i + (int64_t)s * kq];
}

// core = (Z_ab + Z_ba^T) / 2 (q x q), written into the QR work matrix.
struct CoreProb {
  int64_t zab, zba, out;
  int q, ld;
};
__global__ void core_kernel(const CoreProb* __restrict__ cp, int nprob, const double* __restrict__ Z,
                            double* __restrict__ out) {
  int p = blockIdx.y;
  if (p >= nprob) return;
  const CoreProb c = cp[p];
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)c.q * c.q) return;
  int i = (int)(g % c.q), j = (int)(g / c.q);
  out[c.out + g] = 0.5 * (Z[c.zab + i + (int64_t)j * c.ld] + Z[c.zba + j + (int64_t)i * c.ld]);
}

// trace of the leaf diagonal blocks: sum_p H[p, leafpos[p]]
__global__ void diag_trace_kernel(const double* __restrict__ H, const int* __restrict__ leafpos, int64_t n,
                                  int nl, double* __restrict__ part, int df) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x; p < n; p += (int64_t)gridDim.x * 256)
    s += load_val(H + p * nl + leafpos[p], df);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
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
__global__ void unit_cols_kernel(const int* __restrict__ leafpos, int64_t n, int nl, double* __restrict__ E,
                                 int df) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * nl) return;
  int64_t p = g / nl;
  int c = (int)(g % nl);
  store_val(E + g, (c == leafpos[p]) ? 1.0 : 0.0, df);
}
// y = (y + x) / 2
__global__ void average_kernel(double* __restrict__ y, const double* __restrict__ x, int64_t n, int df) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  if (df) {
    float2 a = reinterpret_cast<float2*>(y)[g], b = reinterpret_cast<const float2*>(x)[g];
    df64 v = df_scale(df_add({a.x, a.y}, {b.x, b.y}), 0.5f);
    reinterpret_cast<float2*>(y)[g] = make_float2(v.hi, v.lo);
  } else {
    y[g] = 0.5 * y[g] + 0.5 * x[g];
  }
}

// ----------------------------------------------------------------- host
namespace {

struct PBox {
  int box, start, cnt, slot;
  int nsib;             // number of siblings
  int sib[3];           // indices (into the level's PBox list) of the siblings
  int r[3];             // r_ab for each sibling (U_ab columns)
  int ucol[3];          // column offset of U_ab within Ucat_a
  int Ra;
  int64_t ucat;         // offset of Ucat_a in the pool
  int64_t pcol;         // column offset of this box's block in the P / Q temps
};
struct PPair {
  int a, b;             // a < b (indices into the level's PBox list)
  int sa, sb;           // position of b among a's siblings, a among b's
  int64_t m;            // offset of M_ab (r_ab x r_ba, ld r_ab)
};
struct PLevel {
  int lev = 0;
  std::vector<PBox> bx;
  std::vector<PPair> pr;
  DBuf pool;            // Ucat blocks then M blocks
  int64_t sumRa = 0;
  GemmBatch gP, gQ, gY; // application of G^(lev)
  bool active = false;
};

GemmDesc mk(int M, int N, int K, int8_t abase, int64_t a, int lda, int8_t ta, int8_t bbase, int64_t b, int ldb,
            int8_t tb, int8_t cbase, int64_t c, int ldc, double alpha, double beta, int8_t triB = 0) {
  GemmDesc g{};
  g.M = M; g.N = N; g.K = K;
  g.abase = abase; g.a = a; g.lda = lda; g.ta = ta;
  g.bbase = bbase; g.b = b; g.ldb = ldb; g.tb = tb;
  g.cbase = cbase; g.c = c; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta; g.triB = triB;
  return g;
}

void run_gemm(const std::vector<GemmDesc>& d, double* p0, double* p1, double* p2, double* p3, cudaStream_t s,
              int64_t sc0 = 1, int64_t sc1 = 1, int64_t sc2 = 1, int64_t sc3 = 1, int df = 0) {
  if (d.empty()) return;
  GemmBatch gb;
  gb.build(d, s);
  GemmBases b{};
  b.p[0] = p0; b.p[1] = p1; b.p[2] = p2; b.p[3] = p3;
  b.sc[0] = sc0; b.sc[1] = sc1; b.sc[2] = sc2; b.sc[3] = sc3;
  b.alpha_scale = 1.0;
  b.df = df;
  gb.run(b, s);
}

template <class T>
void upload_prefix(DBuf& d, DBuf& pre, const std::vector<T>& v, const std::vector<int64_t>& prefix,
                   cudaStream_t s) {
  upload(d, v, s);
  upload(pre, prefix, s);
}

// Y -= G^(lev) X for row-major (n x nc) X, Y.
void apply_level(const PLevel& P, const double* X, double* Y, int nc, DBuf& tmp, cudaStream_t s, int df) {
  if (!P.active) return;
  int64_t need = (int64_t)nc * 2 * std::max<int64_t>(1, P.sumRa);
  if ((int64_t)tmp.bytes < need * (int64_t)sizeof(double)) tmp.alloc(need * sizeof(double), s);
  GemmBases b{};
  b.p[0] = const_cast<double*>(X); b.p[1] = Y; b.p[2] = P.pool.as<double>(); b.p[3] = tmp.as<double>();
  b.sc[0] = nc; b.sc[1] = nc; b.sc[2] = 1; b.sc[3] = nc;
  b.M = nc; b.ld = nc; b.alpha_scale = 1.0;
  b.df = df;
  P.gP.run(b, s);
  P.gQ.run(b, s);
  P.gY.run(b, s);
}

// Y -= G^(lev) X for the block-sparse test matrix of a finer level: column
// block k (qc columns) of X is nonzero only on the rows listed in
// slotlist[sb[k] .. sb[k+1]) (ascending tree positions), so the first product
// U_ba^T X(I_b) runs over those rows only.
void apply_level_sparse(const PLevel& P, const double* X, double* Y, int qc, const std::vector<int>& slotlist,
                        const int64_t sb[5], const int* d_slotlist, DBuf& tmp, cudaStream_t s, int df) {
  if (!P.active) return;
  const int nc = 4 * qc;
  int64_t need = (int64_t)nc * 2 * std::max<int64_t>(1, P.sumRa);
  if ((int64_t)tmp.bytes < need * (int64_t)sizeof(double)) tmp.alloc(need * sizeof(double), s);
  std::vector<GemmDesc> g;
  for (const PBox& A : P.bx) {
    if (A.Ra == 0) continue;
    for (int k = 0; k < 4; k++) {
      auto b0 = slotlist.begin() + sb[k], b1 = slotlist.begin() + sb[k + 1];
      auto lo = std::lower_bound(b0, b1, A.start), hi = std::lower_bound(b0, b1, A.start + A.cnt);
      GemmDesc d = mk(qc, A.Ra, (int)(hi - lo), 0, (int64_t)k * qc, nc, 0, 2, A.ucat, A.cnt, 0, 3,
                      A.pcol * nc + (int64_t)k * qc, nc, 1.0, 0.0);
      d.gatherK = 1;
      d.kofs = lo - slotlist.begin();
      d.kb0 = A.start;
      g.push_back(d);
    }
  }
  {
    GemmBatch gb;
    gb.build(g, s);
    GemmBases b{};
    b.p[0] = const_cast<double*>(X); b.p[1] = Y; b.p[2] = P.pool.as<double>(); b.p[3] = tmp.as<double>();
    b.sc[0] = b.sc[1] = b.sc[2] = b.sc[3] = 1;
    b.alpha_scale = 1.0;
    b.df = df;
    b.kidx = d_slotlist;
    gb.run(b, s);
  }
  GemmBases b{};
  b.p[0] = const_cast<double*>(X); b.p[1] = Y; b.p[2] = P.pool.as<double>(); b.p[3] = tmp.as<double>();
  b.sc[0] = nc; b.sc[1] = nc; b.sc[2] = 1; b.sc[3] = nc;
  b.M = nc; b.ld = nc; b.alpha_scale = 1.0;
  b.df = df;
  P.gQ.run(b, s);
  // Y(rows of slot s, column block k)^T -= Q_a(block k)^T Ucat_a(rows, :)^T for
  // k != s only: a box's own-slot samples are never used, and rows outside
  // the level's sibling boxes need none
  std::vector<GemmDesc> gy;
  for (const PBox& A : P.bx) {
    if (A.Ra == 0) continue;
    for (int sl = 0; sl < 4; sl++) {
      auto b0 = slotlist.begin() + sb[sl], b1 = slotlist.begin() + sb[sl + 1];
      auto lo = std::lower_bound(b0, b1, A.start), hi = std::lower_bound(b0, b1, A.start + A.cnt);
      if (hi == lo) continue;
      for (int k = 0; k < 4; k++) {
        if (k == sl) continue;
        GemmDesc d = mk(qc, (int)(hi - lo), A.Ra, 3, (P.sumRa + A.pcol) * nc + (int64_t)k * qc, nc, 0, 2, A.ucat,
                        A.cnt, 1, 1, (int64_t)k * qc, nc, -1.0, 1.0);
        d.gatherN = 1;
        d.nofs = lo - slotlist.begin();
        d.nb0 = A.start;
        gy.push_back(d);
      }
    }
  }
  GemmBatch gb;
  gb.build(gy, s);
  GemmBases c{};
  c.p[0] = const_cast<double*>(X); c.p[1] = Y; c.p[2] = P.pool.as<double>(); c.p[3] = tmp.as<double>();
  c.sc[0] = c.sc[1] = c.sc[2] = c.sc[3] = 1;
  c.alpha_scale = 1.0;
  c.df = df;
  c.kidx = d_slotlist;
  gb.run(c, s);
}

}  // namespace

// Hash of the sparse embedding's choices: SplitMix64 (Steele, Lea & Flood
// 2014) chained over the key (seed, tree position, level, operator, block).
static inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
static inline uint64_t sketch_hash(uint64_t seed, uint64_t pos, int lev, int op, int t) {
  uint64_t h = splitmix64(seed ^ 0x2545F4914F6CDD1Dull);
  h = splitmix64(h ^ pos);
  return splitmix64(h ^ ((uint64_t)lev << 16) ^ ((uint64_t)op << 8) ^ (uint64_t)t);
}

// Peels the traces of up to two symmetric operators together (Sec. 3):
//   operator 0: G_0 = F^-1                          (when want0)
//   operator 1: G_1 = (F^-1 F_k + F_k F^-1) / 2     (when Fk is given)
// Both share every test matrix and sketch, and F^-1 W -- one of the four
// multi-RHS applications G_1 W needs -- is G_0 W, so peeling both costs the
// applications of G_1 alone.
// Rademacher probes for Hutchinson's estimator (Sec. 3, Eq. (hutch)): the
// sign of Philox stream 1's normal draw at (tree position, probe), scaled by
// 1/sqrt(m) so that sums of u^T G u over the m probes are the mean.
__global__ void hutch_probe_kernel(int64_t n, int m, unsigned long long seed, double scale, double* __restrict__ U) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * m) return;
  const int64_t p = g / m;
  const int j = (int)(g % m);
  const double v = philox_normal((unsigned)p, (unsigned)j, 0u, 1u, seed);
  U[g] = v >= 0.0 ? scale : -scale;
}

// Hutchinson's estimator of Tr(F^-1) and Tr(F^-1 F_k) with m probes u:
// mean of u^T F^-1 u and of (F^-1 u)^T (F_k u) (F symmetric), per point set
// (the probes restricted to a set's rows).  One solve and one apply with m
// right-hand sides instead of the peeling's level sweep; its error is
// statistical (standard error ~ sqrt(2/m) ||G||_F).
static void hutch_traces(rsf_handle_s* F, rsf_handle_s* Fk, bool want0, const rsf_opts& o,
                         double* const d_out[2], int64_t d_stride, double* h_sets) {
  cudaStream_t s = F->stream;
  TreeData& T = F->tree_raw->t;
  const int64_t n = T.n;
  const int m = std::max(1, o.probes);
  DBuf U, V, W, res;
  U.alloc(sizeof(double) * n * m, s);
  V.alloc(sizeof(double) * n * m, s);
  LAUNCH(hutch_probe_kernel, cdiv(n * m, 256), 256, 0, s, n, m, (unsigned long long)o.seed, 1.0 / std::sqrt((double)m),
         U.as<double>());
  solve_rows(F, RSF_OP_INV, U.as<double>(), V.as<double>(), m, 0);
  if (Fk) {
    W.alloc(sizeof(double) * n * m, s);
    solve_rows(Fk, RSF_OP_APPLY, U.as<double>(), W.as<double>(), m, 0);
  }
  res.alloc(sizeof(double) * 2 * T.nsets, s);
  res.zero();
  for (int j = 0; j < T.nsets; j++) {
    const int64_t r0 = T.set_off[j], cnt = T.set_off[j + 1] - r0;
    if (want0 || !Fk) dot_into(U.as<double>() + r0 * m, V.as<double>() + r0 * m, cnt * m, res.as<double>() + j, s);
    if (Fk) dot_into(V.as<double>() + r0 * m, W.as<double>() + r0 * m, cnt * m, res.as<double>() + T.nsets + j, s);
  }
  for (int i = 0; i < 2; i++)
    if (d_out[i])
      for (int j = 0; j < T.nsets; j++)
        RSF_CUDA(cudaMemcpyAsync(d_out[i] + (int64_t)j * d_stride, res.as<double>() + i * T.nsets + j, sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
  if (h_sets) {
    d2h(h_sets, res.as<double>(), 2 * T.nsets, s);
    sync(s);
  }
}

void peel_traces(rsf_handle_s* F, rsf_handle_s* Fk, bool want0, double tol, const rsf_opts& o,
                 double* const d_out[2], int64_t d_stride, double* h_sets) {
  if (o.trace_form == RSF_TRACE_HUTCH) {
    hutch_traces(F, Fk, want0, o, d_out, d_stride, h_sets);
    return;
  }
  cudaStream_t s = F->stream;
  TreeData& T = F->tree_raw->t;
  const int64_t n = T.n;
  const int L = T.L;
  const int c_over = std::max(0, o.oversample);
  DevStatus* dst = F->status.as<DevStatus>();
  int64_t n64 = n;
  const int df = F->df;
  std::vector<int> ops;
  if (want0 || !Fk) ops.push_back(0);
  if (Fk) ops.push_back(1);
  const int nops = (int)ops.size();

  // G_o W for the wanted operators, row-major tree-order blocks in F's
  // arithmetic (df64 pairs when F is mixed precision).  Two symmetric forms
  // with the traces of F^-1 and F^-1 F_k:
  //   sym:  G_0 = F^-1,            G_1 = (F^-1 F_k + F_k F^-1) / 2   (Eq. (Gbb))
  //   sqrt: G_0 = F^-1/2 F^-T/2,   G_1 = F^-1/2 F_k F^-T/2
  // (F = F^1/2 F^T/2, so Tr(F^-1/2 F_k F^-T/2) = Tr(F^-T/2 F^-1/2 F_k)).
  const bool sqrt_form = o.trace_form == RSF_TRACE_SQRT;
  DBuf ga, gb2, gw;
  // sp (may be null): the column-block structure of a test matrix, whose
  // first solves (F^-1 W, F_k W) then skip the zero blocks
  auto applyG = [&](const double* in, double* const out[2], int q, const SparseRHS* sp) {
    const int64_t cnt = n64 * q;
    const int64_t bytes = sizeof(double) * cnt;
    // doubles in and out when F is df64 but F_k is fp64
    const bool split = Fk && df && !Fk->df;
    const int io = split ? 0 : df;
    const double* x = in;
    if (split) {
      if ((int64_t)gw.bytes < bytes) gw.alloc(bytes, s);
      RSF_CUDA(cudaMemcpyAsync(gw.p, in, bytes, cudaMemcpyDeviceToDevice, s));
      convert_df64(gw.as<double>(), cnt, 0, s);
      x = gw.as<double>();
    }
    if ((int64_t)ga.bytes < bytes) ga.alloc(bytes, s);
    if (sqrt_form) {
      solve_rows(F, RSF_OP_INV_SQRT_T, x, ga.as<double>(), q, io);        // F^-T/2 W
      if (want0 || !Fk) solve_rows(F, RSF_OP_INV_SQRT, ga.as<double>(), out[0], q, io);
      if (Fk) {
        if ((int64_t)gb2.bytes < bytes) gb2.alloc(bytes, s);
        solve_rows(Fk, RSF_OP_APPLY, ga.as<double>(), gb2.as<double>(), q, io);
        solve_rows(F, RSF_OP_INV_SQRT, gb2.as<double>(), out[1], q, io);   // F^-1/2 F_k F^-T/2 W
      }
    } else {
      if (!Fk) {
        solve_rows(F, RSF_OP_INV, x, out[0], q, io, sp);
        return;
      }
      if ((int64_t)gb2.bytes < bytes) gb2.alloc(bytes, s);
      double* x3 = want0 ? out[0] : gb2.as<double>();
      // G_1 W is only read outside each box's own slot block (the sample
      // blocks Y_ab take the siblings' slots), so the outer solves skip it
      solve_rows(F, RSF_OP_INV, x, x3, q, io, sp);                        // F^-1 W
      solve_rows(Fk, RSF_OP_APPLY, x3, out[1], q, io, nullptr, sp);       // F_k F^-1 W
      solve_rows(Fk, RSF_OP_APPLY, x, ga.as<double>(), q, io, sp);
      double* x2 = want0 ? gb2.as<double>() : x3;
      solve_rows(F, RSF_OP_INV, ga.as<double>(), x2, q, io, nullptr, sp); // F^-1 F_k W
      LAUNCH(average_kernel, cdiv(cnt, 256), 256, 0, s, out[1], x2, cnt, io);
    }
    if (split)
      for (int oi : ops) convert_df64(out[oi], cnt, 1, s);
  };

  std::vector<PLevel> levels[2];
  levels[0].resize(L + 1);
  levels[1].resize(L + 1);
  DBuf tmpP;  // P/Q temps for apply_level
  std::vector<int> slotrow(n);
  DBuf dslot;
  int r_prev[2] = {0, 0};

  for (int lev = 1; lev <= L; lev++) {
    PLevel TL;  // the level's boxes and sibling pairs (shared by both operators)
    TL.lev = lev;
    std::vector<int> idx_of(T.level.size(), -1);
    for (int b : T.by_level[lev]) {
      int par = T.parent[b];
      int nsib = 0;
      for (int sl = 0; sl < 4; sl++) nsib += T.children[par][sl] >= 0;
      if (nsib < 2) continue;
      PBox pb{};
      pb.box = b; pb.start = T.start[b]; pb.cnt = T.count[b]; pb.slot = T.slot[b];
      idx_of[b] = (int)TL.bx.size();
      TL.bx.push_back(pb);
    }
    if (TL.bx.empty()) continue;
    for (auto& pb : TL.bx) {
      int par = T.parent[pb.box];
      pb.nsib = 0;
      for (int sl = 0; sl < 4; sl++) {
        int c = T.children[par][sl];
        if (c >= 0 && c != pb.box) pb.sib[pb.nsib++] = idx_of[c];
      }
    }
    for (int a = 0; a < (int)TL.bx.size(); a++)
      for (int t = 0; t < TL.bx[a].nsib; t++) {
        int b = TL.bx[a].sib[t];
        if (a < b) {
          PPair pp{};
          pp.a = a; pp.b = b; pp.sa = t;
          for (int u = 0; u < TL.bx[b].nsib; u++)
            if (TL.bx[b].sib[u] == a) pp.sb = u;
          TL.pr.push_back(pp);
        }
      }
    const int nbx = (int)TL.bx.size();
    std::fill(slotrow.begin(), slotrow.end(), -1);
    for (auto& pb : TL.bx)
      for (int i = 0; i < pb.cnt; i++) slotrow[pb.start + i] = pb.slot;
    upload(dslot, slotrow, s);
    // rows of each slot in tree order (the nonzero rows of W_k)
    std::vector<int> slotlist;
    int64_t sbeg[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 4; k++) {
      sbeg[k] = (int64_t)slotlist.size();
      for (int64_t p = 0; p < n64; p++)
        if (slotrow[p] == k) slotlist.push_back((int)p);
    }
    sbeg[4] = (int64_t)slotlist.size();
    DBuf dslotlist;
    upload(dslotlist, slotlist, s);
    // column-block structure of this level's test matrices on every level
    // >= lev: a box's rows are nonzero only in its level-lev ancestor's slot
    SparseRHS sparse;
    sparse.lev0 = lev;
    sparse.slot.assign(F->levels.size(), {});
    for (int l = lev; l < (int)F->levels.size(); l++) {
      const std::vector<int>& bl = F->levels[l].box;
      sparse.slot[l].assign(bl.size(), -1);
      for (size_t i = 0; i < bl.size(); i++) {
        int a = bl[i];
        while (T.level[a] > lev) a = T.parent[a];
        if (idx_of[a] >= 0) sparse.slot[l][i] = T.slot[a];
      }
    }

    // ordered pairs (a, t): box a with its t-th sibling
    struct OPair { int a, t; };
    std::vector<OPair> op;
    for (int a = 0; a < nbx; a++)
      for (int t = 0; t < TL.bx[a].nsib; t++) op.push_back({a, t});
    const int nop = (int)op.size();
    std::vector<int> opbase(nbx + 1, 0);
    for (int a = 0; a < nbx; a++) opbase[a + 1] = opbase[a] + TL.bx[a].nsib;
    auto opidx = [&](int a, int t) { return opbase[a] + t; };

    // Per-operator sample counts.  Initial guess: at level 1 nine tenths of
    // the largest level-1 skeleton of F (the sibling-block ranks at eps_peel
    // sit below the ID ranks at eps_fact); below, the operator's largest rank
    // on the previous level times a per-level factor.  The factors follow the
    // rank profiles measured for Matern 3/2 on clustered points at n = 65,536
    // and 262,144 (from level 2 to 3 the ranks grow by up to 1.2x, deeper
    // levels shrink them by 0.35-0.85x per level); a short guess costs a
    // second sketch and QR of the level, a long one surplus columns, and the
    // adaptive retry below keeps the result independent of the guess.
    // The applications are shared: the columns drawn are those of the
    // operator that needs the most, and each operator compresses with the
    // first q_o of them (the columns are i.i.d., so any prefix is itself a
    // valid test matrix).
    auto level_factor = [](int l) {
      return l <= 2 ? 0.9 : l == 3 ? 1.25 : l == 4 ? 0.85 : l == 5 ? 0.75 : l <= 7 ? 0.7 : 0.6;
    };
    struct OpState {
      int qo = 0;
      bool done = true;
      std::vector<int> rank;
      QRBatch qb;
      DBuf Yb, Sb, Sqr;
      std::vector<int64_t> yoff, soff;
    };
    OpState st[2];
    for (int oi : ops) {
      int g = 8;
      if (lev == 1) {
        g = std::max(o.q0, 1);
        if (F->levels.size() > 1)
          for (int kk : F->levels[1].k) g = std::max(g, (9 * kk) / 10);
      } else {
        g = std::max(g, (int)(level_factor(lev) * r_prev[oi]));
      }
      st[oi].qo = g + c_over;
      st[oi].done = false;
      st[oi].rank.assign(nop, 0);
      st[oi].yoff.assign(nop + 1, 0);
      st[oi].soff.assign(nop + 1, 0);
    }
    const int qcap = (int)std::min<int64_t>(n64, 1 << 15);
    if (verbose()) {
      int kf = 0, kfp = 0;
      if ((int)F->levels.size() > lev)
        for (int kk : F->levels[lev].k) kf = std::max(kf, kk);
      if (lev > 1 && (int)F->levels.size() > lev - 1)
        for (int kk : F->levels[lev - 1].k) kfp = std::max(kfp, kk);
      fprintf(stderr, "[rsf] peel level %d: largest skeleton of F %d (level above %d), previous ranks %d %d\n", lev, kf,
              kfp, r_prev[0], r_prev[1]);
    }
    std::vector<int> chunk_q, chunk_col0;
    std::vector<DBuf> Wch, Ych[2];
    DBuf WV;
    std::vector<int64_t> woff(nbx + 1, 0);
    int qtot = 0;
    while (true) {
      int q = qtot;
      for (int oi : ops)
        if (!st[oi].done) q = std::max(q, st[oi].qo);
      if (q > qtot) {
        const int qc = q - qtot;
        DBuf Wn, Y[2];
        Wn.alloc(sizeof(double) * n64 * 4 * qc, s);
        for (int oi : ops) Y[oi].alloc(sizeof(double) * n64 * 4 * qc, s);
        LAUNCH(gen_w_kernel, cdiv(n64 * 4 * qc, 256), 256, 0, s, dslot.as<int>(), n64, qc, qtot, lev,
               (unsigned long long)o.seed, Wn.as<double>(), df);
        int tk = prof_begin(s);
        double* const outs[2] = {Y[0].as<double>(), Y[1].as<double>()};
        sparse.qc = qc;
        applyG(Wn.as<double>(), outs, 4 * qc, &sparse);
        prof_end(tk, s, PROF_PEEL_APPLY, 0, 0);
        tk = prof_begin(s);
        for (int oi : ops)
          if (!st[oi].done)
            for (int m = 1; m < lev; m++)
              apply_level_sparse(levels[oi][m], Wn.as<double>(), Y[oi].as<double>(), qc, slotlist, sbeg,
                                 dslotlist.as<int>(), tmpP, s, df);
        prof_end(tk, s, PROF_PEEL_SUB, 0, 0);
        chunk_q.push_back(qc);
        chunk_col0.push_back(qtot);
        Wch.push_back(std::move(Wn));
        for (int oi : ops) Ych[oi].push_back(std::move(Y[oi]));
        qtot = q;
        // W_a (|I_a| x q) per box, column-major: the box's rows of its slot's
        // test columns
        for (int a = 0; a < nbx; a++) woff[a + 1] = woff[a] + (int64_t)TL.bx[a].cnt * q;
        WV.alloc(sizeof(double) * std::max<int64_t>(1, woff[nbx]), s);
        for (size_t ch = 0; ch < Wch.size(); ch++) {
          int qq = chunk_q[ch];
          std::vector<ExtractProb> ew;
          std::vector<int64_t> pw(1, 0);
          for (int a = 0; a < nbx; a++) {
            const PBox& A = TL.bx[a];
            ew.push_back({(int64_t)A.start, woff[a], A.cnt, A.slot * qq});
            pw.push_back(pw.back() + (int64_t)A.cnt * qq);
          }
          DBuf d3, d4;
          upload_prefix(d3, d4, ew, pw, s);
          LAUNCH(extract_kernel, cdiv(pw.back(), 256), 256, 0, s, d3.as<ExtractProb>(), d4.as<int64_t>(), nbx,
                 pw.back(), qq, 4 * qq, chunk_col0[ch], Wch[ch].as<double>(), WV.as<double>(), 0);
        }
      }
      int tq = prof_begin(s);
      bool all_done = true;
      for (int oi : ops) {
        OpState& S = st[oi];
        if (S.done) continue;
        const int qo = S.qo;
        // Y_ab (|I_a| x q_o) per ordered pair, column-major, in the arithmetic
        // of the applications (df64 or fp64)
        for (int i = 0; i < nop; i++) S.yoff[i + 1] = S.yoff[i] + (int64_t)TL.bx[op[i].a].cnt * qo;
        for (int i = 0; i < nop; i++) S.soff[i + 1] = S.soff[i] + (int64_t)qo * qo;
        S.Yb.alloc(sizeof(double) * std::max<int64_t>(1, S.yoff[nop]), s);
        for (size_t ch = 0; ch < Wch.size(); ch++) {
          const int qq = chunk_q[ch];
          const int take = std::min(qq, qo - chunk_col0[ch]);
          if (take <= 0) continue;
          std::vector<ExtractProb> ey;
          std::vector<int64_t> py(1, 0);
          for (int i = 0; i < nop; i++) {
            const PBox& A = TL.bx[op[i].a];
            const PBox& Bx = TL.bx[A.sib[op[i].t]];
            ey.push_back({(int64_t)A.start, S.yoff[i], A.cnt, Bx.slot * qq});
            py.push_back(py.back() + (int64_t)A.cnt * take);
          }
          DBuf d1, d2;
          upload_prefix(d1, d2, ey, py, s);
          LAUNCH(extract_kernel, cdiv(py.back(), 256), 256, 0, s, d1.as<ExtractProb>(), d2.as<int64_t>(), nop,
                 py.back(), take, 4 * qq, chunk_col0[ch], Ych[oi][ch].as<double>(), S.Yb.as<double>(), 0);
        }
        // Z_ab = W_a(:, :q_o)^T Y_ab (q_o x q_o, for the core of Eq.
        // (lowrankapprox)).  The
        // rank-revealing QR runs on Y_ab itself when the box has at most 2 q_o
        // rows, else on a sparse sign embedding Omega_a Y_ab of Y_ab into
        // ell = 2 q_o rows (rounded up to a multiple of SKETCH_S): every row of
        // the box is added, with a random sign, to one random row in each of
        // SKETCH_S blocks of ell / SKETCH_S rows (an OSNAP embedding, Nelson &
        // Nguyen 2013), independent of the test matrices.
        std::vector<char> direct(nop);
        for (int i = 0; i < nop; i++) direct[i] = TL.bx[op[i].a].cnt <= 2 * qo;
        S.Sb.alloc(sizeof(double) * std::max<int64_t>(1, S.soff[nop]), s);
        {
          std::vector<GemmDesc> g;
          for (int i = 0; i < nop; i++) {
            const PBox& A = TL.bx[op[i].a];
            g.push_back(mk(qo, qo, A.cnt, 0, woff[op[i].a], A.cnt, 1, 1, S.yoff[i], A.cnt, 0, 2, S.soff[i], qo,
                           1.0, 0.0));
          }
          run_gemm(g, WV.as<double>(), S.Yb.as<double>(), S.Sb.as<double>(), nullptr, s, 1, 1, 1, 1, df);
          if (df) convert_df64(S.Sb.as<double>(), S.soff[nop], 0, s);
        }
        const int bsz = (2 * qo + SKETCH_S - 1) / SKETCH_S;
        const int ell = bsz * SKETCH_S;
        // rank-revealing pivoted QR (fp64): the blocks taken from Y_ab first
        // (one contiguous range, converted from df64 in place), then the
        // ell x q_o sketches
        std::vector<int> qrows(nop);
        std::vector<int64_t> qoff(nop, 0);
        int64_t ndirect = 0, nqr = 0;
        for (int i = 0; i < nop; i++) {
          qrows[i] = direct[i] ? TL.bx[op[i].a].cnt : ell;
          if (direct[i]) { qoff[i] = nqr; nqr += (int64_t)qrows[i] * qo; }
        }
        ndirect = nqr;
        for (int i = 0; i < nop; i++)
          if (!direct[i]) { qoff[i] = nqr; nqr += (int64_t)qrows[i] * qo; }
        S.Sqr.alloc(sizeof(double) * std::max<int64_t>(1, nqr), s);
        {
          std::vector<CopyProb> cy;
          for (int i = 0; i < nop; i++)
            if (direct[i]) cy.push_back({qrows[i], qo, qrows[i], qrows[i], S.yoff[i], qoff[i], 0});
          if (!cy.empty()) {
            copy_batched(cy, S.Yb.as<double>(), S.Sqr.as<double>(), s);
            if (df) convert_df64(S.Sqr.as<double>(), ndirect, 0, s);
          }
          // the embedding of every sketched box: per bucket (row of Omega_a)
          // the list of (box row, sign), ordered by box row
          std::vector<int> bucket_of_box(nbx, -1);
          std::vector<int> bptr(1, 0), ent;
          for (int i = 0; i < nop; i++) {
            const int a = op[i].a;
            if (direct[i] || bucket_of_box[a] >= 0) continue;
            const PBox& A = TL.bx[a];
            bucket_of_box[a] = (int)bptr.size() - 1;
            std::vector<int> cnt(ell + 1, 0), hu((size_t)A.cnt * SKETCH_S);
            std::vector<char> neg((size_t)A.cnt * SKETCH_S);
            for (int r = 0; r < A.cnt; r++)
              for (int t = 0; t < SKETCH_S; t++) {
                const uint64_t h = sketch_hash(o.seed, (uint64_t)(A.start + r), lev, oi, t);
                const int u = t * bsz + (int)(h % (uint64_t)bsz);
                hu[(size_t)r * SKETCH_S + t] = u;
                neg[(size_t)r * SKETCH_S + t] = (char)(h >> 63);
                cnt[u + 1]++;
              }
            for (int u = 0; u < ell; u++) cnt[u + 1] += cnt[u];
            const int base = (int)ent.size();
            ent.resize(base + (size_t)A.cnt * SKETCH_S);
            std::vector<int> fill(cnt.begin(), cnt.end() - 1);
            for (int r = 0; r < A.cnt; r++)
              for (int t = 0; t < SKETCH_S; t++) {
                const size_t k = (size_t)r * SKETCH_S + t;
                ent[base + fill[hu[k]]++] = (r << 1) | neg[k];
              }
            for (int u = 1; u <= ell; u++) bptr.push_back(base + cnt[u]);
          }
          std::vector<SketchProb> sk;
          for (int i = 0; i < nop; i++) {
            if (direct[i]) continue;
            const PBox& A = TL.bx[op[i].a];
            sk.push_back({S.yoff[i], qoff[i], A.cnt, bucket_of_box[op[i].a]});
          }
          if (!sk.empty()) {
            DBuf dsk, dbp, den;
            upload(dsk, sk, s);
            upload(dbp, bptr, s);
            upload(den, ent, s);
            const int64_t total = (int64_t)sk.size() * ell * qo;
            LAUNCH(sparse_sketch_kernel, cdiv(total, 256), 256, 0, s, dsk.as<SketchProb>(), total, ell, qo,
                   dbp.as<int>(), den.as<int>(), S.Yb.as<double>(), S.Sqr.as<double>(), df);
          }
        }
        std::vector<QRProb> qp(nop);
        for (int i = 0; i < nop; i++) {
          qp[i] = QRProb{};
          qp[i].m = qrows[i]; qp[i].c = qo; qp[i].cpiv = qo; qp[i].maxk = qo;
          qp[i].lda = std::max(1, qrows[i]); qp[i].a = qoff[i]; qp[i].tol = tol;
        }
        S.qb = QRBatch();
        S.qb.build(qp, s);
        S.qb.run(S.Sqr.as<double>(), dst, lev, s);
        std::vector<QRState> hst(nop);
        d2h(hst.data(), S.qb.d_state(), nop, s);
        sync(s);
        int rm = 0;
        for (int i = 0; i < nop; i++) {
          S.rank[i] = hst[i].k;
          rm = std::max(rm, S.rank[i]);
        }
        if (verbose())
          fprintf(stderr, "[rsf] peel op %d level %d: q %d, max rank %d, pairs %d, boxes %d\n", oi, lev, qo, rm, nop,
                  nbx);
        if (rm <= qo - c_over || qo >= qcap) {
          S.done = true;
        } else {
          // saturated: grow geometrically; otherwise just past the detected rank
          if (rm >= qo - 1) S.qo = std::max(qo + c_over, (4 * qo) / 3);
          else S.qo = rm + c_over + std::max(4, rm / 16);
          S.qo = std::min(S.qo, qcap);
          all_done = false;
        }
      }
      prof_end(tq, s, PROF_PEEL_QR, 0, 0);
      if (all_done) break;
    }
    Wch.clear();
    for (int oi : ops) Ych[oi].clear();
    WV.release();
    for (int oi : ops) {
      OpState& S = st[oi];
      PLevel& PL = levels[oi][lev];
      PL.lev = lev;
      PL.bx = TL.bx;
      PL.pr = TL.pr;
      PL.active = true;
      const int q = S.qo;
      std::vector<int>& rank = S.rank;
      std::vector<int64_t>& yoff = S.yoff;
      std::vector<int64_t>& soff = S.soff;
      QRBatch& qb = S.qb;
      DBuf& Yb = S.Yb;
      DBuf& Sb = S.Sb;
      DBuf& Sqr = S.Sqr;
      int& rp = r_prev[oi];
      // a block whose row or column space is empty is dropped in both directions
      for (const PPair& pp : PL.pr) {
        int iab = opidx(pp.a, pp.sa), iba = opidx(pp.b, pp.sb);
        if (rank[iab] == 0 || rank[iba] == 0) rank[iab] = rank[iba] = 0;
      }
      rp = 0;
      for (int i = 0; i < nop; i++) rp = std::max(rp, rank[i]);

      int trest = prof_begin(s);
      // ---- pool layout: U_ab blocks (Ucat_a per box), then the cores M_ab
      int64_t pool = 0;
      PL.sumRa = 0;
      for (int i = 0; i < nop; i++) PL.bx[op[i].a].r[op[i].t] = rank[i];
      for (int a = 0; a < nbx; a++) {
        PBox& A = PL.bx[a];
        A.Ra = 0;
        for (int t = 0; t < A.nsib; t++) { A.ucol[t] = A.Ra; A.Ra += A.r[t]; }
        A.ucat = pool;
        pool += (int64_t)A.cnt * A.Ra;
        A.pcol = PL.sumRa;
        PL.sumRa += A.Ra;
      }
      const int64_t mstart = pool;
      for (auto& pp : PL.pr) {
        pp.m = pool;
        pool += (int64_t)PL.bx[pp.a].r[pp.sa] * PL.bx[pp.b].r[pp.sb];
      }
      PL.pool.alloc(sizeof(double) * std::max<int64_t>(1, pool), s);
      PL.pool.zero();
      double* UP = PL.pool.as<double>();
      // ---- R11^-1 of every sketch QR, U_ab = Y_ab(:, piv) R11^-1 and
      //      B_ab = W_a^T U_ab = Z_ab(:, piv) R11^-1 with Z_ab = W_a^T Y_ab
      std::vector<int64_t> roff(nop + 1, 0), poff(nop + 1, 0), zpoff(nop + 1, 0), boff(nop + 1, 0);
      for (int i = 0; i < nop; i++) {
        int rows = PL.bx[op[i].a].cnt;
        roff[i + 1] = roff[i] + (int64_t)rank[i] * rank[i];
        poff[i + 1] = poff[i] + (int64_t)rows * rank[i];
        zpoff[i + 1] = zpoff[i] + (int64_t)q * rank[i];
        boff[i + 1] = boff[i] + (int64_t)q * rank[i];
      }
      DBuf Rinv, Ypiv, Zpiv, Bm;
      Rinv.alloc(sizeof(double) * std::max<int64_t>(1, roff[nop]), s);
      {
        std::vector<TrsmProb> tp(nop);
        for (int i = 0; i < nop; i++) tp[i] = {rank[i], -1, roff[i]};
        qr_trsm(qb, tp, nullptr, Sqr.as<double>(), Rinv.as<double>(), dst, lev, s);
      }
      Ypiv.alloc(sizeof(double) * std::max<int64_t>(1, poff[nop]), s);
      Zpiv.alloc(sizeof(double) * std::max<int64_t>(1, zpoff[nop]), s);
      Bm.alloc(sizeof(double) * std::max<int64_t>(1, boff[nop]), s);
      {
        std::vector<PivGather> pg(nop), pz(nop);
        std::vector<int64_t> gp(nop + 1, 0), gz(nop + 1, 0);
        for (int i = 0; i < nop; i++) {
          int rows = PL.bx[op[i].a].cnt;
          pg[i] = {yoff[i], poff[i], qb.colprefix_h[i], rows, rows};
          pz[i] = {soff[i], zpoff[i], qb.colprefix_h[i], q, q};
          gp[i + 1] = gp[i] + (int64_t)rows * rank[i];
          gz[i + 1] = gz[i] + (int64_t)q * rank[i];
        }
        if (gp[nop] > 0) {
          DBuf d1, d2, d3, d4;
          upload_prefix(d1, d2, pg, gp, s);
          LAUNCH(pivgather_kernel, cdiv(gp[nop], 256), 256, 0, s, d1.as<PivGather>(), d2.as<int64_t>(), nop,
                 gp[nop], qb.d_piv(), qb.d_state(), Yb.as<double>(), Ypiv.as<double>());
          upload_prefix(d3, d4, pz, gz, s);
          LAUNCH(pivgather_kernel, cdiv(gz[nop], 256), 256, 0, s, d3.as<PivGather>(), d4.as<int64_t>(), nop,
                 gz[nop], qb.d_piv(), qb.d_state(), Sb.as<double>(), Zpiv.as<double>());
        }
        std::vector<GemmDesc> gu, gb;
        for (int i = 0; i < nop; i++) {
          const PBox& A = PL.bx[op[i].a];
          int r = rank[i];
          if (r == 0) continue;
          // U = Ypiv (rows x r) * Rinv (r x r, upper) into Ucat_a
          gu.push_back(mk(A.cnt, r, r, 0, poff[i], A.cnt, 0, 1, roff[i], r, 0, 2,
                          A.ucat + (int64_t)A.ucol[op[i].t] * A.cnt, A.cnt, 1.0, 0.0, 2));
          // B = Zpiv (q x r) * Rinv
          gb.push_back(mk(q, r, r, 0, zpoff[i], q, 0, 1, roff[i], r, 0, 2, boff[i], q, 1.0, 0.0, 2));
        }
        // both products in the arithmetic of the applications; B returns to
        // fp64 for the least-squares QRs of the cores
        if (df) {
          convert_df64(Rinv.as<double>(), roff[nop], 1, s);
          convert_df64(Zpiv.as<double>(), zpoff[nop], 1, s);
        }
        run_gemm(gb, Zpiv.as<double>(), Rinv.as<double>(), Bm.as<double>(), nullptr, s, 1, 1, 1, 1, df);
        if (df) convert_df64(Bm.as<double>(), boff[nop], 0, s);
        run_gemm(gu, Ypiv.as<double>(), Rinv.as<double>(), UP, nullptr, s, 1, 1, 1, 1, df);
      }
      Ypiv.release();
      Yb.release();
      // ---- cores M_ab (Eq. (lowrankapprox))
      {
        const int npr = (int)PL.pr.size();
        // X1 = (B_ab)^+ core  via QR of [B_ab | core]  (q x (r_ab + q))
        std::vector<QRProb> q1;
        std::vector<CopyProb> cp1;
        std::vector<CoreProb> cores;
        std::vector<int> live;
        int64_t qpool = 0;
        for (int p = 0; p < npr; p++) {
          const PPair& pp = PL.pr[p];
          int iab = opidx(pp.a, pp.sa), iba = opidx(pp.b, pp.sb);
          int rab = rank[iab], rba = rank[iba];
          if (rab == 0 || rba == 0) continue;
          live.push_back(p);
          QRProb x{};
          x.m = q; x.c = rab + q; x.cpiv = rab; x.maxk = rab; x.lda = q; x.a = qpool; x.tol = 0.0;
          cp1.push_back({q, rab, q, q, boff[iab], qpool, 0});
          cores.push_back({soff[iab], soff[iba], qpool + (int64_t)q * rab, q, q});
          qpool += (int64_t)q * (rab + q);
          q1.push_back(x);
        }
        if (!live.empty()) {
          DBuf W1;
          W1.alloc(sizeof(double) * qpool, s);
          copy_batched(cp1, Bm.as<double>(), W1.as<double>(), s);
          {
            DBuf dc;
            upload(dc, cores, s);
            dim3 grid(cdiv((int64_t)q * q, 256), (unsigned)cores.size());
            LAUNCH(core_kernel, grid, 256, 0, s, dc.as<CoreProb>(), (int)cores.size(), Sb.as<double>(), W1.as<double>());
          }
          QRBatch qx;
          qx.build(q1, s);
          qx.run(W1.as<double>(), dst, lev, s);
          std::vector<int> rhs;
          std::vector<TrsmProb> tp(live.size());
          std::vector<int64_t> toff(live.size() + 1, 0);
          std::vector<PermScatter> ps(live.size());
          std::vector<int64_t> xoff(live.size() + 1, 0), spre(live.size() + 1, 0);
          for (size_t j = 0; j < live.size(); j++) {
            const PPair& pp = PL.pr[live[j]];
            int rab = rank[opidx(pp.a, pp.sa)];
            tp[j].nrhs = q;
            tp[j].rhs0 = (int64_t)rhs.size();
            tp[j].out0 = toff[j];
            for (int t = 0; t < q; t++) rhs.push_back(rab + t);
            toff[j + 1] = toff[j] + (int64_t)rab * q;
            // X1 (r_ab x q, ld r_ab): X1[piv[i], s] = t[i, s]
            ps[j] = {toff[j], xoff[j], qx.colprefix_h[j], rab, q, 1, rab};
            xoff[j + 1] = xoff[j] + (int64_t)rab * q;
            spre[j + 1] = spre[j] + (int64_t)rab * q;
          }
          DBuf drhs, tout, X1;
          upload(drhs, rhs, s);
          tout.alloc(sizeof(double) * std::max<int64_t>(1, toff.back()), s);
          X1.alloc(sizeof(double) * std::max<int64_t>(1, xoff.back()), s);
          X1.zero();
          qr_trsm(qx, tp, drhs.as<int>(), W1.as<double>(), tout.as<double>(), dst, lev, s);
          {
            DBuf d1, d2;
            upload_prefix(d1, d2, ps, spre, s);
            LAUNCH(permscatter_kernel, cdiv(spre.back(), 256), 256, 0, s, d1.as<PermScatter>(), d2.as<int64_t>(),
                   (int)ps.size(), spre.back(), qx.d_piv(), qx.d_state(), tout.as<double>(), X1.as<double>());
          }
          // M_ab^T = (B_ba)^+ X1^T via QR of [B_ba | X1^T]  (q x (r_ba + r_ab))
          std::vector<QRProb> q2;
          std::vector<CopyProb> cp2, cpx;
          int64_t qpool2 = 0;
          for (size_t j = 0; j < live.size(); j++) {
            const PPair& pp = PL.pr[live[j]];
            int iab = opidx(pp.a, pp.sa), iba = opidx(pp.b, pp.sb);
            int rab = rank[iab], rba = rank[iba];
            QRProb x{};
            x.m = q; x.c = rba + rab; x.cpiv = rba; x.maxk = rba; x.lda = q; x.a = qpool2; x.tol = 0.0;
            cp2.push_back({q, rba, q, q, boff[iba], qpool2, 0});
            cpx.push_back({q, rab, rab, q, xoff[j], qpool2 + (int64_t)q * rba, 1});
            qpool2 += (int64_t)q * (rba + rab);
            q2.push_back(x);
          }
          DBuf W2;
          W2.alloc(sizeof(double) * qpool2, s);
          copy_batched(cp2, Bm.as<double>(), W2.as<double>(), s);
          copy_batched(cpx, X1.as<double>(), W2.as<double>(), s);
          QRBatch qy;
          qy.build(q2, s);
          qy.run(W2.as<double>(), dst, lev, s);
          std::vector<int> rhs2;
          std::vector<TrsmProb> tp2(live.size());
          std::vector<int64_t> toff2(live.size() + 1, 0), spre2(live.size() + 1, 0);
          std::vector<PermScatter> ps2(live.size());
          for (size_t j = 0; j < live.size(); j++) {
            const PPair& pp = PL.pr[live[j]];
            int rab = rank[opidx(pp.a, pp.sa)], rba = rank[opidx(pp.b, pp.sb)];
            tp2[j].nrhs = rab;
            tp2[j].rhs0 = (int64_t)rhs2.size();
            tp2[j].out0 = toff2[j];
            for (int t = 0; t < rab; t++) rhs2.push_back(rba + t);
            toff2[j + 1] = toff2[j] + (int64_t)rba * rab;
            // M^T[piv[i], s] = t[i, s]  ->  M (r_ab x r_ba, ld r_ab): M[s, piv[i]]
            ps2[j] = {toff2[j], pp.m, qy.colprefix_h[j], rba, rab, rab, 1};
            spre2[j + 1] = spre2[j] + (int64_t)rba * rab;
          }
          DBuf drhs2, tout2;
          upload(drhs2, rhs2, s);
          tout2.alloc(sizeof(double) * std::max<int64_t>(1, toff2.back()), s);
          qr_trsm(qy, tp2, drhs2.as<int>(), W2.as<double>(), tout2.as<double>(), dst, lev, s);
          {
            DBuf d1, d2;
            upload_prefix(d1, d2, ps2, spre2, s);
            LAUNCH(permscatter_kernel, cdiv(spre2.back(), 256), 256, 0, s, d1.as<PermScatter>(), d2.as<int64_t>(),
                   (int)ps2.size(), spre2.back(), qy.d_piv(), qy.d_state(), tout2.as<double>(), UP);
          }
        }
      }
      if (df) convert_df64(UP + mstart, pool - mstart, 1, s);
      // ---- application descriptors of G^(lev) (bases 0 X, 1 Y, 2 pool, 3 temp)
      {
        std::vector<GemmDesc> gP, gQ, gY;
        for (int a = 0; a < nbx; a++) {
          const PBox& A = PL.bx[a];
          if (A.Ra == 0) continue;
          // P_a^T (nc x Ra) = X(I_a)^T Ucat_a
          gP.push_back(mk(-1, A.Ra, A.cnt, 0, A.start, -1, 0, 2, A.ucat, A.cnt, 0, 3, A.pcol, -1, 1.0, 0.0));
          // Y(I_a)^T -= Q_a^T Ucat_a^T, Q stored after all P blocks
          gY.push_back(mk(-1, A.cnt, A.Ra, 3, PL.sumRa + A.pcol, -1, 0, 2, A.ucat, A.cnt, 1, 1, A.start, -1, -1.0,
                          1.0));
        }
        for (const PPair& pp : PL.pr) {
          const PBox& A = PL.bx[pp.a];
          const PBox& Bx = PL.bx[pp.b];
          int rab = A.r[pp.sa], rba = Bx.r[pp.sb];
          if (rab == 0 || rba == 0) continue;
          // Q_ab^T (nc x r_ab) = P_(b->a)^T (nc x r_ba) M_ab^T
          gQ.push_back(mk(-1, rab, rba, 3, Bx.pcol + Bx.ucol[pp.sb], -1, 0, 2, pp.m, rab, 1, 3,
                          PL.sumRa + A.pcol + A.ucol[pp.sa], -1, 1.0, 0.0));
          // Q_ba^T (nc x r_ba) = P_(a->b)^T (nc x r_ab) M_ab
          gQ.push_back(mk(-1, rba, rab, 3, A.pcol + A.ucol[pp.sa], -1, 0, 2, pp.m, rab, 0, 3,
                          PL.sumRa + Bx.pcol + Bx.ucol[pp.sb], -1, 1.0, 0.0));
        }
        PL.gP.build(gP, s);
        PL.gQ.build(gQ, s);
        PL.gY.build(gY, s);
      }
      prof_end(trest, s, PROF_PEEL_REST, 0, 0);
      Sqr.release();
      Sb.release();
    }
    sync(s);
  }

  // ---- extraction: H = (G - sum_m G^(m)) E, trace of the leaf blocks
  const int nl = std::max(1, T.max_leaf);
  const DBuf& dlp = T.leafpos_d;
  DBuf E, H[2];
  E.alloc(sizeof(double) * n64 * nl, s);
  for (int oi : ops) H[oi].alloc(sizeof(double) * n64 * nl, s);
  LAUNCH(unit_cols_kernel, cdiv(n64 * nl, 256), 256, 0, s, dlp.as<int>(), n64, nl, E.as<double>(), df);
  int tk = prof_begin(s);
  double* const hout[2] = {H[0].as<double>(), H[1].as<double>()};
  applyG(E.as<double>(), hout, nl, nullptr);
  prof_end(tk, s, PROF_PEEL_APPLY, 0, 0);
  tk = prof_begin(s);
  for (int oi : ops)
    for (int m = 1; m <= L; m++) apply_level(levels[oi][m], E.as<double>(), H[oi].as<double>(), nl, tmpP, s, df);
  prof_end(tk, s, PROF_PEEL_SUB, 0, 0);
  // the trace of every point set: its rows are contiguous in tree order
  const int nsets = T.nsets;
  DBuf part, res;
  part.alloc(sizeof(double) * 1024, s);
  res.alloc(sizeof(double) * 2 * nsets, s);
  for (int oi : ops) {
    for (int si = 0; si < nsets; si++) {
      const int64_t r0 = T.set_off[si], cnt = T.set_off[si + 1] - r0;
      const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, cdiv(cnt, 256)));
      LAUNCH(diag_trace_kernel, nb, 256, 0, s, H[oi].as<double>() + r0 * nl, dlp.as<int>() + r0, cnt, nl,
             part.as<double>(), df);
      double* outp = d_out[oi] ? d_out[oi] + si * d_stride : res.as<double>() + oi * nsets + si;
      LAUNCH(sum_parts_kernel, 1, 256, 0, s, part.as<double>(), nb, outp);
      if (h_sets) d2h(&h_sets[oi * nsets + si], outp, 1, s);
    }
  }
  sync(s);
}

}  // namespace rsf
