// Batched ragged fp64 dense linear algebra used by every level of the
// factorization, the solves and the peeling: GEMM, column-pivoted Householder
// QR (one launch pair per elimination step over all problems), triangular
// solves and a blocked Cholesky.
#pragma once

#include "common.cuh"

namespace rsf {

// C = alpha op(A) op(B) + beta C, column-major.  Pointers are offsets into
// one of four base arrays passed at launch, so descriptor arrays built once
// can be reused with fresh buffers (M < 0 / ld < 0 take the launch's values).
struct GemmDesc {
  int M, N, K;
  int lda, ldb, ldc;
  int64_t a, b, c;
  int8_t abase, bbase, cbase;
  int8_t ta, tb;
  int8_t triB;   // 0: none, 1: op(B) lower triangular, 2: op(B) upper triangular
  int8_t lowC;   // 1: skip output tiles strictly above the diagonal
  int8_t gatherK;  // 1: the K index runs over kidx[kofs .. kofs + K): A column
                   //    (ta = 0) kidx[.], B row (tb = 0) kidx[.] - kb0
  double alpha, beta;
  int64_t kofs;
  int64_t kb0;
  int8_t gatherN;  // 1: the N index runs over kidx[nofs .. nofs + N): B row
                   //    of op(B) (tb = 1) kidx[.] - nb0, C column kidx[.]
  int64_t nofs;
  int64_t nb0;
  int m0;          // first row of A and C (ta = 0): the M range [m0, m0 + M)
                   // of a wider column-major operand, e.g. one column block
                   // of a row-major multi-RHS block
};

// Output-tile shape (rows, columns) of the tensor-core GEMM kernels, the K
// chunk of one stage and the superblock of K terms summed in the tensor
// memory between two epilogues of the pre-sliced engine.
constexpr int TC_BM = 128;
constexpr int TC_BN = 64;
constexpr int TC_KC = 16;
constexpr int TC_SBK = 384;

// Index of the problem owning tile `tile` given the per-problem tile prefix.
__device__ __forceinline__ int find_prob(const int* prefix, int nprob, int tile) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct GemmBases {
  double* p[4];
  int64_t sc[4];  // offset multiplier per base (row-major buffers: the row length)
  int M;       // used where desc.M < 0
  int ld;      // used where desc.lda/ldc < 0
  double alpha_scale;  // multiplies every desc.alpha
  int df;              // nonzero: operands and result are df64 pairs (df64.cuh),
                       // multiplied on the tensor cores (1: pre-sliced operands
                       // in work buffers; 3: sliced inside the GEMM kernel, no
                       // work buffers; tcgemm.cu) or in df64 arithmetic on the
                       // CUDA cores (2)
  const int* kidx;     // K index list of descriptors with gatherK
};

// Plan of the pre-sliced tensor-core engine (tcgemm.cu) for one descriptor:
// its K in 16-term chunks (nch) and 384-term superblocks (nsb), and the
// offsets before it of its slicing work items (pi + qi * mtL), A slice
// blocks (pa + qa * mtL) and A exponents (pe + qe * mtL), where mtL is the
// launch's number of 128-row tiles (the q parts count descriptors whose M
// is the launch's).
struct TcDescPlan {
  int nch, nsb;
  int64_t pi, qi, pa, qa, pe, qe;
};
// The same for one (descriptor, 64-column tile) entry: offsets of its B
// slice blocks, B exponents and slicing work items.
struct TcEntryPlan {
  int64_t bblk, be, pib;
};

// Device-resident batch of GEMM problems with its tile prefix.
struct GemmBatch {
  DBuf desc, prefix, ntile_tc;
  // TcDescPlan per descriptor, TcEntryPlan per ntile_tc entry: built with the
  // batch, uploaded at the first launch on the pre-sliced engine
  mutable DBuf tc_dplan, tc_eplan;
  mutable std::vector<TcDescPlan> tc_dplan_h;
  mutable std::vector<TcEntryPlan> tc_eplan_h;
  // totals of the plans (fixed part, launch-M part per M-tile)
  int64_t tc_pi = 0, tc_qi = 0, tc_pa = 0, tc_qa = 0, tc_pe = 0, tc_qe = 0, tc_bblk = 0, tc_be = 0, tc_pib = 0;
  int nprob = 0;
  int ntilesN = 0;   // sum over problems of ceil(N / BN)
  int ntilesN_tc = 0; // the same for the TC_BN-column tiles of the tensor-core
                      // kernel, whose (problem, first column) pairs ntile_tc lists
  int maxM = 0;      // max M over problems with M >= 0
  bool anyLaunchM = false;
  // algorithmic work: flops = 2 (fixedMNK + launchM * launchNK), same for bytes
  double fixedMNK = 0, launchNK = 0, fixedBytes = 0, launchBytesPerM = 0, launchBytes0 = 0;
  void build(const std::vector<GemmDesc>& d, cudaStream_t s);
  void run(const GemmBases& b, cudaStream_t s) const;
};

// Tensor-core (tcgen05) engine for df64 batches (tcgemm.cu): runs g with
// the launch's largest M; tc_status_take returns and clears the engine's
// device status (RSF_ETIMEOUT when a bounded wait gave up).
void tc_gemm_run(const GemmBatch& g, const GemmBases& b, int M, cudaStream_t s);
// Pre-sliced tensor-core engine (tcgemm.cu): slices every operand once into
// stream-ordered work buffers, then multiplies; the default for df64 batches.
void tc_gemm_pre_run(const GemmBatch& g, const GemmBases& b, int M, cudaStream_t s);
int tc_status_take();
void gemm_selftest(int engine, int m, int n, int k, int ta, int tb, double alpha, const double* A, int lda,
                   const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s);
void convert_df64(double* p, int64_t n, int to, cudaStream_t s);
// Batches whose largest M is below this run on the CUDA-core df64 kernel
// (a 128-row tensor-core tile would be mostly empty).
constexpr int TC_MIN_M = 64;

// ----------------------------------------------------------- pivoted QR
// One problem: A (m x c, column-major, leading dimension lda) at offset a of
// the QR pool.  Only the first cpiv columns may be pivots; the others are
// carried along (they receive Q^T).  Stops after maxk steps or when the next
// pivot's column norm is <= tol * (first pivot norm) (tol > 0).
struct QRProb {
  int m, c, cpiv, maxk, lda;
  int64_t a;        // offset of A in the pool
  int64_t col0;     // offset of this problem's per-column arrays (size c)
  int64_t row0;     // offset of this problem's Householder vector (size m)
  double tol;
};
struct QRState {
  int done, k, pad0, pad1;
  double r11, tau;
  unsigned long long key[2];
};

struct QRBatch {
  int nprob = 0;
  int64_t ncols = 0, nrows = 0;
  int maxsteps = 0;
  std::vector<int> colprefix_h;   // host copy of the column prefix (for launch sizing)
  DBuf prob, state, piv, chosen, vbuf, colprefix, colprob, ndone, nu2, nuref2;
  // m (rows) may be finalised on the device (near-field counts) before run().
  void build(const std::vector<QRProb>& p, cudaStream_t s);
  // Runs all steps; pool is the matrix storage; st is the status word.
  void run(double* pool, DevStatus* st, int level, cudaStream_t s);
  int* d_piv() const { return piv.as<int>(); }
  QRState* d_state() const { return state.as<QRState>(); }
  QRProb* d_prob() const { return prob.as<QRProb>(); }
};

// After a QR with truncation: per problem, the [S, R] permutation (S = pivot
// order, R = remaining eligible columns in increasing order) written to
// perm[out0 .. out0 + cpiv) and k to kout.
void qr_split(const QRBatch& qb, const int64_t* d_out0, int* d_perm, int* d_kout, cudaStream_t s);

// Runs the QR kernel's grid barrier so that its bounded wait must give up
// (one participant more than launched); returns the device status code
// (RSF_ETIMEOUT when the limit works).  Takes a few seconds.
int barrier_timeout_selftest(cudaStream_t s);

// Back-substitution with the QR's upper triangle R11 (k x k, pivot order):
// for each problem and each right-hand side column listed by rhs (physical
// column indices of A, count nrhs per problem), solve R11 t = A[0:k, col]
// into out (k x nrhs column-major at out0, ld k).  Identity mode (rhs null):
// right-hand sides are the unit vectors e_0..e_{k-1} (gives R11^-1).
struct TrsmProb {
  int nrhs;
  int64_t rhs0;   // offset into the rhs column-index array (or -1: identity)
  int64_t out0;   // offset of the output in outpool
};
void qr_trsm(const QRBatch& qb, const std::vector<TrsmProb>& tp, const int* d_rhs,
             double* pool, double* outpool, DevStatus* st, int level, cudaStream_t s);

// ----------------------------------------------------------- Cholesky
// In place lower Cholesky of n x n blocks (column-major, ld) at offsets a in
// pool; upper triangles are left untouched (garbage).  Blocked: one panel
// kernel per 32 columns plus a lower-triangle GEMM for the trailing matrix.
struct CholProb {
  int n, ld;
  int64_t a;
  int box;       // reported on failure
};
void cholesky_batched(const std::vector<CholProb>& p, double* pool, DevStatus* st,
                      int level, cudaStream_t s);

// Inverse of lower-triangular blocks: out (n x n, ld n, zero upper) at outoff
// from in (n x n at a, ld) -- one warp per column.
struct TriInvProb {
  int n, ld;
  int64_t a, out;
};
void lower_inverse_batched(const std::vector<TriInvProb>& p, const double* in,
                           double* out, cudaStream_t s);

// Symmetrise square blocks: A <- (A + A^T) / 2.
struct SqProb {
  int n, ld;
  int64_t a;
};
void symmetrize_batched(const std::vector<SqProb>& p, double* pool, cudaStream_t s);

// Copy sub-blocks: dst[i + j*ldd] = src[i + j*lds] (or transposed source).
struct CopyProb {
  int m, n, lds, ldd;
  int64_t src, dst;
  int trans;  // 1: dst[i + j*ldd] = src[j + i*lds]
};
void copy_batched(const std::vector<CopyProb>& p, const double* src, double* dst, cudaStream_t s);

}  // namespace rsf
