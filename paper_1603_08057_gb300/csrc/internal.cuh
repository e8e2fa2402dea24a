// Internal structures of the RSF library (tree, factorization levels) and
// the device kernel-function evaluation shared by the assembly kernels.
#pragma once

#include <array>
#include <memory>

#include "dense.cuh"

struct rsf_tree_s;
struct rsf_handle_s;

namespace rsf {

constexpr int DEPTH_BITS = 24;
// A derivative factorization keeps its df64 solve factors when a df64 apply
// agrees with the fp64 apply to this multiple of the ID tolerance.
constexpr double DF64_APPLY_TOL_FACTOR = 10.0;

struct KernelParams {
  int family;
  double alpha;
  double l, s2, nug;
  int which;  // 0 Sigma, 1 d/dl (d/dl1), 2 d/ds2, 3 d/dnug, 4 d/dl2
  int aniso;  // scaled distance of Sec. 5.1 with length scales l (x) and l2 (y)
  double l2;
};

// Modified Bessel functions K0(x), K1(x) for x > 0 in fp64, for the Matern
// kernel with nu = 1.  For x < 1 the ascending series (Abramowitz & Stegun
// 9.6.13 and 9.6.11 with n = 1; ten terms reach 1e-16), otherwise the
// integral K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the
// trapezoid rule, which converges exponentially for this analytic,
// doubly decaying integrand: step h = min(1/4, 1/(2 sqrt x)) (the integrand's
// width shrinks like x^-1/2), cut where x (cosh t - 1) > 40 (terms below
// e^-40 of the first); 13 to 18 terms for x in [1, 80], relative error below
// 5e-14 against reference values.  cosh(kh) by the recurrence
// cosh((k+1)h) = 2 cosh(h) cosh(kh) - cosh((k-1)h).
__device__ __forceinline__ void bessel_k01(double x, double& k0, double& k1) {
  const double euler_gamma = 0.57721566490153286061;
  if (x < 1.0) {
    const double y = 0.25 * x * x;
    double t0 = 1.0, t1 = 1.0, H = 0.0;
    double i0 = 1.0, s0 = 0.0, i1s = 1.0, s1 = -2.0 * euler_gamma + 1.0;   // k = 0 terms
    for (int k = 1; k < 12; k++) {
      t0 *= y / ((double)k * k);
      t1 *= y / ((double)k * (k + 1));
      H += 1.0 / k;
      i0 += t0;
      s0 += H * t0;
      i1s += t1;
      s1 += (2.0 * (H - euler_gamma) + 1.0 / (k + 1)) * t1;
    }
    const double lx = log(0.5 * x);
    k0 = -(lx + euler_gamma) * i0 + s0;
    k1 = 1.0 / x + lx * (0.5 * x * i1s) - 0.25 * x * s1;
    return;
  }
  const double h = fmin(0.25, 0.5 / sqrt(x));
  const double u = 1.0 + 40.0 / x;
  const int n = (int)ceil(log(u + sqrt(u * u - 1.0)) / h);
  const double ch = 0.5 * (exp(h) + exp(-h));
  double c_prev = ch, c = 1.0;   // cosh(-h), cosh(0)
  const double e0 = exp(-x);
  double s0 = 0.5 * e0, s1 = 0.5 * e0;
  for (int k = 1; k <= n; k++) {
    const double cn = 2.0 * ch * c - c_prev;
    c_prev = c;
    c = cn;
    const double e = exp(-x * c);
    s0 += e;
    s1 += e * c;
  }
  k0 = h * s0;
  k1 = h * s1;
}

// Off-diagonal entry of Sigma (which 0) or dSigma/dtheta (which 1, 2, 3) at
// distance r (Sec. 1 Eqs. (matern), (rationalquadratic); Sec. 5.5).
__device__ __forceinline__ double kernel_offdiag(const KernelParams& kp, double r) {
  if (kp.which == 3) return 0.0;
  const double l = kp.l;
  double k, dk;  // correlation and its l-derivative
  switch (kp.family) {
    case RSF_MATERN12: {
      double e = exp(-r / l);
      k = e;
      dk = (r / (l * l)) * e;
      break;
    }
    case RSF_MATERN32: {
      double a = 1.7320508075688772 * r / l;
      double e = exp(-a);
      k = (1.0 + a) * e;
      dk = a * a * e / l;
      break;
    }
    case RSF_MATERN52: {
      double a = 2.23606797749979 * r / l;
      double e = exp(-a);
      k = (1.0 + a + a * a / 3.0) * e;
      dk = (a * a / 3.0) * (1.0 + a) * e / l;
      break;
    }
    case RSF_MATERN1: {
      // x K1(x) and, with (x K1)' = -x K0, d/dl = x^2 K0(x) / l
      const double x = 1.4142135623730951 * r / l;
      if (x < 1e-300) {
        k = 1.0;
        dk = 0.0;
      } else {
        double b0, b1;
        bessel_k01(x, b0, b1);
        k = x * b1;
        dk = x * x * b0 / l;
      }
      break;
    }
    default: {  // RSF_RQ
      double u = 1.0 + r * r / (2.0 * kp.alpha * l * l);
      double p = pow(u, -kp.alpha);
      k = p;
      dk = p / u * r * r / (l * l * l);
      break;
    }
  }
  if (kp.which == 0) return kp.s2 * k;
  if (kp.which == 1) return kp.s2 * dk;
  return k;
}

__device__ __forceinline__ double kernel_diag(const KernelParams& kp) {
  if (kp.which == 0) return kp.s2 + kp.nug;
  if (kp.which == 1 || kp.which == 4) return 0.0;
  return 1.0;
}

__device__ __forceinline__ double dist2(double ax, double ay, double bx, double by) {
  double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Off-diagonal entry between points a and b.  Isotropic: the family at the
// Euclidean distance.  Anisotropic (Sec. 5.1): the family at unit length
// scale on r = ||a - b||_theta, u = (ax - bx)/l, v = (ay - by)/l2,
// r^2 = u^2 + v^2; as the correlation depends on r only, its l- and
// l2-derivatives are k'(r) dr/dl with dr/dl = -u^2/(l r) (and v^2/(l2 r) for
// l2), and k'(r) = -(unit-length l-derivative)/r, so the entry is the
// unit-length l-derivative times u^2/(l r^2) (resp. v^2/(l2 r^2)).
__device__ __forceinline__ double kernel_pair(const KernelParams& kp, double ax, double ay, double bx, double by) {
  if (!kp.aniso) return kernel_offdiag(kp, sqrt(dist2(ax, ay, bx, by)));
  if (kp.which == 3) return 0.0;
  const double u = __dsub_rn(ax, bx) / kp.l, v = __dsub_rn(ay, by) / kp.l2;
  const double r2 = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
  const double r = sqrt(r2);
  KernelParams k1 = kp;
  k1.l = 1.0;
  if (kp.which == 0 || kp.which == 2) return kernel_offdiag(k1, r);
  if (r2 == 0.0) return 0.0;
  k1.which = 1;
  const double w = kp.which == 1 ? u * u / kp.l : v * v / kp.l2;
  return kernel_offdiag(k1, r) * (w / r2);
}

// Host view of the quadtree (Sec. 2.1, Remark (tree)); device copies of the
// tree-order coordinates and permutation.
struct TreeData {
  int64_t n = 0;
  double lo[2] = {0, 0}, side = 1.0;
  int n_occ = 64;
  int L = 0;
  // boxes (root first, levels contiguous)
  std::vector<int> level, start, count, parent, slot, ix, iy;
  std::vector<std::array<int, 4>> children;
  std::vector<char> is_leaf;
  std::vector<double> cx, cy, w;
  std::vector<std::vector<int>> by_level;
  DBuf leafpos_d;                // device: per tree position, index in its leaf
  int max_leaf = 0;
  // independent point sets (batched datasets): set i holds tree positions
  // [set_off[i], set_off[i+1]) and has its own root square
  int nsets = 1;
  std::vector<int64_t> set_off;
  std::vector<double> set_lo, set_side;   // 2 and 1 per set
  std::vector<int> box_set;               // set of every box
  DBuf box_set_d;                         // device copies of box_set and set_off
  DBuf set_off_d;
  cudaStream_t stream = nullptr;
  DBuf xt;     // n x 2 tree-order coordinates
  DBuf perm;   // tree position -> original index (int)
  DBuf iperm;  // original index -> tree position (int)
};

// One level of the factorization (boxes processed together).
struct LevelData {
  int lev = 0;
  int nb = 0;
  std::vector<int> box;                 // tree box ids
  std::vector<int> c, k, r;             // |I|, |S|, |R|
  std::vector<int64_t> row0;            // row offset of the box in the level's row space
  int64_t nrows = 0;                    // sum of c
  std::vector<int64_t> toff, eoff, doff, dioff;  // factor pool offsets: T, E, D, Dinv
  std::vector<char> leafbox;
  DBuf fpool;    // this level's factor storage (T, E, D, Dinv)
  DBuf rr;       // per box R-row range (first row, count) for the middle copies
  int nrr = 0;
  DBuf Isr;      // DOF ids (tree positions) in [S, R] order, nrows ints
  DBuf src;      // gather map: >= 0 row of level lev+1, < 0: -(1 + tree position)
  // solve descriptors (offset based; bases: 0 = X in, 1 = X out/tmp, 2 = factor pool)
  GemmBatch gRS_T;   // X_R += a * (op T) X_S   (C = R rows, A = S rows, B = T)
  GemmBatch gSR_Et;  // X_S += a * E X_R
  GemmBatch gRS_E;   // X_R += a * E^T X_S
  GemmBatch gSR_Tt;  // X_S += a * T X_R
  // middle (block diagonal) products on R rows: out = in * op(B)
  GemmBatch gMid[5];  // 0: Dinv^T, 1: Dinv, 2: D, 3: D^T, 4: D (full, indefinite)
  // host copies of the descriptors above and the level box index of each
  // (for solves whose right-hand sides are column-block sparse)
  std::vector<GemmDesc> hRS_T, hSR_Et, hRS_E, hSR_Tt, hMid[5];
  std::vector<int> boxRSE, boxMid[5];
};

}  // namespace rsf

// Opaque handle types of the C ABI.
struct rsf_tree_s {
  rsf::TreeData t;
  rsf_opts opts;
};

struct rsf_handle_s {
  std::shared_ptr<rsf_tree_s> tree;   // shared with other handles built on it
  rsf_tree_s* tree_raw = nullptr;
  rsf::KernelParams kp;
  rsf_opts opts;
  double tol = 0;
  bool spd = true;
  int df = 0;                          // solve factors: 0 fp64; df64 pairs multiplied on the
                                       // tensor cores (1) or on the CUDA cores (2)
  cudaStream_t stream = nullptr;
  int device = -1;                     // CUDA device current when the handle was built
  std::vector<rsf::LevelData> levels;  // index = tree level (0 = root)
  rsf::DBuf status;                    // DevStatus
  rsf::DBuf logdet_parts;              // per box partial log-determinants
  int64_t nboxes_total = 0;
  // bookkeeping
  int max_rank = 0, max_active = 0;
  double flops = 0, kevals = 0;
  int64_t factor_entries = 0;
  double probe_rel_diff = -1;          // derivative factorization: df64 vs fp64 apply (-1: no probe)
};

namespace rsf {
// A forest over independent point sets: set_off (host, nsets + 1 prefix
// offsets into points) -- one set gives the plain quadtree.
std::shared_ptr<rsf_tree_s> build_forest(const double* points, const std::vector<int64_t>& set_off,
                                         const rsf_opts& o, cudaStream_t s);
std::shared_ptr<rsf_tree_s> build_tree(const double* points, int64_t n, const rsf_opts& o,
                                       cudaStream_t s);
void factorize(rsf_handle_s* h);
void check_status(rsf_handle_s* h);
// Internal solve on tree-order, row-major (n x q) buffers: out = op(F) in.
// io_df: in/out hold df64 pairs (else doubles, converted when h->df).
// Column-block sparse right-hand sides: the n x q input holds blocks of qc
// columns, and on every level l >= lev0 the rows of level box i are nonzero
// only in block slot[l][i] (-1: nowhere).  The upward sweep and the middle
// factor, which keep that pattern, then run on one block per box.
// The same structure describes outputs of which a box's rows are needed
// only outside block slot[l][i] (on levels >= lev0): the middle factor and
// the downward sweep then skip that block.
struct SparseRHS {
  int lev0 = 0;
  int qc = 0;
  std::vector<std::vector<int>> slot;   // per level, per level box
};
void solve_rows(rsf_handle_s* h, int op, const double* in, double* out, int q, int io_df = 0,
                const SparseRHS* sp = nullptr, const SparseRHS* skip_out = nullptr);
// In-place conversion of n doubles to df64 pairs (to = 1) or back (to = 0).
void convert_df64(double* p, int64_t n, int to, cudaStream_t s);
// Peeled traces (Sec. 3) of G_0 = F^-1 (when want0 or Fk is null) and of
// G_1 = (F^-1 Fk + Fk F^-1)/2 (when Fk is given), sharing every test matrix.
// Operator i's trace over point set j goes to d_out[i][j * d_stride] (device,
// d_out[i] may be null) and to h_sets[i * nsets + j] (host, may be null).
void peel_traces(rsf_handle_s* F, rsf_handle_s* Fk, bool want0, double tol, const rsf_opts& o,
                 double* const d_out[2], int64_t d_stride, double* h_sets);
// r = z - Sigma x in tree order (exact kernel, on the fly; df64 for the
// Matern families unless force_fp64), and y += x.
void kernel_residual(rsf_handle_s* F, const double* zt, const double* x, double* rt, int force_fp64 = 0);
void add_into(double* y, const double* x, int64_t n, cudaStream_t s);
// y = K(xs, x) v (kernel kp, no nugget): m new points xs against n points x,
// both device row-major m x 2 / n x 2, v and y device (the conditional
// mean's matvec).
void cross_matvec(KernelParams kp, const double* x, const double* v, int64_t n, const double* xs, int64_t m,
                  double* y, cudaStream_t s);
// Whether kernel_residual runs in df64 for these kernel parameters.
bool residual_uses_df64(const KernelParams& kp);
// Iterative-refinement sweeps of Sigma^-1 z that gp_loglik runs for handle F.
int refine_sweeps(const rsf_handle_s* F);
// device reductions
double dot_device(const double* a, const double* b, int64_t n, cudaStream_t s);
// a . b into a device scalar (stream ordered, no synchronisation)
void dot_into(const double* a, const double* b, int64_t n, double* d_out, cudaStream_t s);
}  // namespace rsf
