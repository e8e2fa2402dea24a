// C ABI (include/rsf.h): argument checks, handle management, the
// log-likelihood (Algorithm 1, first part) and the score (Algorithm 1, loop
// over theta) on top of the factorization, solve and peeling drivers.
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>

#include "internal.cuh"

namespace rsf {

int64_t g_launches = 0;

namespace {
thread_local std::string g_err;

struct Exception {
  rsf_status code;
  std::string msg;
};
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }

// ------------------------------------------------------ kernel timing
namespace {
struct ProfRec {
  cudaEvent_t a, b;
  int cat;
  double flops, bytes;
};
bool g_prof_on = false;
int g_prof_next = 0;
std::map<int, ProfRec> g_prof_open;   // begun, not yet ended (token -> record)
std::vector<ProfRec> g_prof_done;     // ended, not yet read
std::vector<cudaEvent_t> g_event_pool;
struct ProfAcc {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
} g_prof_acc[PROF_NCAT];

cudaEvent_t get_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  RSF_CUDA(cudaEventCreate(&e));
  return e;
}
void prof_drain() {
  for (auto& r : g_prof_done) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ProfAcc& acc = g_prof_acc[r.cat];
      acc.launches++;
      acc.ms += ms;
      acc.flops += r.flops;
      acc.bytes += r.bytes;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof_done.clear();
}
}  // namespace

bool prof_enabled() { return g_prof_on; }

bool verbose() {
  static const bool v = std::getenv("RSF_VERBOSE") != nullptr;
  return v;
}

int prof_begin(cudaStream_t s) {
  if (!g_prof_on) return -1;
  if (g_prof_done.size() > 20000) prof_drain();
  ProfRec r{get_event(), get_event(), -1, 0, 0};
  RSF_CUDA(cudaEventRecord(r.a, s));
  int tok = g_prof_next++ & 0x3fffffff;
  g_prof_open[tok] = r;
  return tok;
}

void prof_end(int token, cudaStream_t s, int cat, double flops, double bytes) {
  if (token < 0) return;
  auto it = g_prof_open.find(token);
  if (it == g_prof_open.end()) return;
  ProfRec r = it->second;
  g_prof_open.erase(it);
  RSF_CUDA(cudaEventRecord(r.b, s));
  r.cat = cat;
  r.flops = flops;
  r.bytes = bytes;
  g_prof_done.push_back(r);
}

void fail(rsf_status code, const std::string& msg) { throw Exception{code, msg}; }

static std::mutex g_hook_mu;
static AllocHook g_hook;
AllocHook alloc_hook() {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  return g_hook;
}

// Trees handed out through the C ABI; handles share ownership.
static std::mutex g_tree_mu;
static std::map<rsf_tree_s*, std::shared_ptr<rsf_tree_s>> g_trees;

// z (user order, device, n x q column-major ld) <-> tree-order row-major.
__global__ void to_tree_kernel(const double* __restrict__ B, int64_t ldb, int q, const int* __restrict__ perm,
                               int64_t n, double* __restrict__ X) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * q) return;
  int64_t p = g / q;
  int c = (int)(g % q);
  X[g] = B[(int64_t)perm[p] + (int64_t)c * ldb];
}
__global__ void from_tree_kernel(const double* __restrict__ X, int64_t n, int q, const int* __restrict__ perm,
                                 double* __restrict__ B, int64_t ldb) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * q) return;
  int64_t p = g / q;
  int c = (int)(g % q);
  B[(int64_t)perm[p] + (int64_t)c * ldb] = X[g];
}

// Scalars slots
// S_Q0.. the quadratic terms and S_R0.. the traces of the p score
// components (l, s2, nug and, anisotropic, l2), S_G0.. the score.
enum { S_QUAD = 0, S_LOGDET, S_LOGLIK, S_AA, S_QL, S_QF, S_QL2, S_TNUG, S_TL, S_TL2,
       S_G0, S_G1, S_G2, S_G3, S_Q0, S_Q1, S_Q2, S_Q3, S_R0, S_R1, S_R2, S_R3,
       S_ONEA, S_ONEB, S_PQ, S_NSLOTS };

// Every point set (one for a plain quadtree, several for batched datasets)
// has its own block of S_NSLOTS scalars.

// Eq. (loglikelihood) per set: l = -quad/2 - log|F|/2 - n/2 log(2 pi)
__global__ void loglik_kernel(double* sc, const int64_t* __restrict__ set_off, int nsets) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsets) return;
  double* c = sc + (int64_t)i * S_NSLOTS;
  double n = (double)(set_off[i + 1] - set_off[i]);
  c[S_LOGLIK] = -0.5 * c[S_QUAD] - 0.5 * c[S_LOGDET] - 0.5 * n * log(2.0 * 3.141592653589793);
}

// Eq. (gradient) per set, with Sigma = s2 Sigma_s2 + nug I:
//   g_l   = (a^T F_l a - Tr_l)/2
//   g_s2  = ((a^T F a - nug a^T a) - (n - nug Tr(F^-1)))/(2 s2)
//   g_nug = (a^T a - Tr(F^-1))/2
//   g_l2  = (a^T F_l2 a - Tr_l2)/2       (anisotropic, p = 4)
__global__ void score_kernel(double* sc, const int64_t* __restrict__ set_off, int nsets, double s2, double nug,
                             int p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsets) return;
  double* c = sc + (int64_t)i * S_NSLOTS;
  double n = (double)(set_off[i + 1] - set_off[i]);
  const double q[4] = {c[S_QL], (c[S_QF] - nug * c[S_AA]) / s2, c[S_AA], c[S_QL2]};
  const double t[4] = {c[S_TL], (n - nug * c[S_TNUG]) / s2, c[S_TNUG], c[S_TL2]};
  for (int k = 0; k < p; k++) {
    c[S_Q0 + k] = q[k];
    c[S_R0 + k] = t[k];
    c[S_G0 + k] = 0.5 * q[k] - 0.5 * t[k];
  }
}

// Profile likelihood, Sec. 5.5 Eq. (prof), with A = Sigma + 1 1^T per set.
// gamma = A^-1 z = alpha - beta (1^T alpha) / (1 + 1^T beta) (Sherman-Morrison)
// from alpha = Sigma^-1 z and beta = Sigma^-1 1 of the row's set.
__global__ void profile_gamma_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                     const int64_t* __restrict__ set_off, int nsets, const double* __restrict__ sc,
                                     double* __restrict__ g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nsets - 1;  // the set holding row i: last k with set_off[k] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (set_off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  const double* c = sc + (int64_t)lo * S_NSLOTS;
  g[i] = a[i] - b[i] * (c[S_ONEA] / (1.0 + c[S_ONEB]));
}

// Eq. (prof) per set with the constant read as n/2 (log n - 1 - log 2 pi):
//   lt   = -log|F|/2 - n/2 log(z^T gamma) + n/2 (log n - 1 - log 2 pi)
//   gt_k = -Tr(Sigma^-1 Sigma_k)/2 + n/2 (gamma^T Sigma_k gamma) / (z^T gamma)
// with gamma's quadratic terms and the traces in S_Q0.., S_R0.. (score_kernel).
__global__ void profile_kernel(double* sc, const int64_t* __restrict__ set_off, int nsets, int with_score, int p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsets) return;
  double* c = sc + (int64_t)i * S_NSLOTS;
  const double n = (double)(set_off[i + 1] - set_off[i]);
  const double qt = c[S_PQ];
  c[S_LOGLIK] = -0.5 * c[S_LOGDET] - 0.5 * n * log(qt) + 0.5 * n * (log(n) - 1.0 - log(2.0 * 3.141592653589793));
  if (with_score)
    for (int k = 0; k < p; k++) c[S_G0 + k] = -0.5 * c[S_R0 + k] + 0.5 * n * c[S_Q0 + k] / qt;
}

__global__ void fill_kernel(double* __restrict__ p, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Two tree-order vectors a, b <-> one n x 2 row-major block X (the layout of
// solve_rows' right-hand sides): X[2i] = a[i], X[2i + 1] = b[i].
__global__ void pack2_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                             double* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    X[2 * i] = a[i];
    X[2 * i + 1] = b[i];
  }
}
__global__ void unpack2_kernel(const double* __restrict__ X, int64_t n, double* __restrict__ a,
                               double* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a[i] = X[2 * i];
    b[i] = X[2 * i + 1];
  }
}

// Conditional samples (Remark conditional): S(:, j) = mean + Y(0:m, j) - P(0:m, j)
__global__ void cond_combine_kernel(const double* __restrict__ mean, const double* __restrict__ Y, int64_t ldy,
                                    const double* __restrict__ P, int64_t ldp, int64_t m, int q,
                                    double* __restrict__ S, int64_t lds) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * q) return;
  const int64_t i = t % m, j = t / m;
  S[i + j * lds] = mean[i] + Y[i + j * ldy] - P[i + j * ldp];
}

// log|F| of every set = sum of its boxes' parts (fixed order; one block per
// set, boxes of other sets skipped)
__global__ void sum_logdet_kernel(const double* __restrict__ parts, const int* __restrict__ box_set, int n,
                                  double* __restrict__ out, int64_t stride) {
  __shared__ double red[256];
  const int set = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256)
    if (box_set[i] == set) s += parts[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)set * stride] = red[0];
}

// rsf_solve with its work buffers in the library's fixed scratch (noalloc.cu).
void solve_noalloc(rsf_handle_s* h, double* B, int64_t ldb, int nrhs, int op);

// Two trees are interchangeable when their box tables and point orders agree
// (e.g. built twice from the same points).
static bool same_tree(rsf_tree_s* a, rsf_tree_s* b) {
  if (a == b) return true;
  const TreeData &A = a->t, &B = b->t;
  if (A.n != B.n || A.start != B.start || A.count != B.count || A.level != B.level) return false;
  std::vector<int> pa(A.n), pb(B.n);
  d2h(pa.data(), A.perm.as<int>(), A.n, A.stream);
  d2h(pb.data(), B.perm.as<int>(), B.n, B.stream);
  sync(A.stream);
  sync(B.stream);
  return pa == pb;
}

static rsf_opts resolve_opts(const rsf_opts* o) {
  rsf_opts r;
  rsf_opts_default(&r);
  if (o) r = *o;
  RSF_CHECK(r.trace_form == RSF_TRACE_SYM || r.trace_form == RSF_TRACE_SQRT || r.trace_form == RSF_TRACE_HUTCH,
            RSF_EINVAL, "trace_form must be RSF_TRACE_SYM, RSF_TRACE_SQRT or RSF_TRACE_HUTCH");
  RSF_CHECK(r.trace_form != RSF_TRACE_HUTCH || (r.probes >= 1 && r.probes <= 65536), RSF_EINVAL,
            "probes must be in 1 .. 65536");
  RSF_CHECK(r.refine >= -1 && r.refine <= 8, RSF_EINVAL, "refine must be in -1 .. 8");
  return r;
}

static void check_kernel(const rsf_kernel* k, const double* theta) {
  RSF_CHECK(k != nullptr && theta != nullptr, RSF_EINVAL, "kernel and theta must not be NULL");
  RSF_CHECK(k->family == RSF_MATERN12 || k->family == RSF_MATERN32 || k->family == RSF_MATERN52 ||
                k->family == RSF_MATERN1 || k->family == RSF_RQ,
            RSF_EINVAL, "unsupported kernel family");
  RSF_CHECK(k->family != RSF_RQ || k->alpha > 0.0, RSF_EINVAL, "RQ needs alpha > 0");
  RSF_CHECK(theta[0] > 0.0 && theta[1] > 0.0 && theta[2] >= 0.0, RSF_EINVAL, "theta must satisfy l > 0, s2 > 0, nug >= 0");
  RSF_CHECK(k->anisotropic == 0 || k->anisotropic == 1, RSF_EINVAL, "anisotropic must be 0 or 1");
  RSF_CHECK(!k->anisotropic || theta[3] > 0.0, RSF_EINVAL, "anisotropic theta needs l2 > 0");
}

// Number of score components: (l, s2, nug), and l2 for anisotropic kernels.
static int nparams(const rsf_kernel* k) { return k->anisotropic ? 4 : 3; }

static rsf_handle_s* make_handle(std::shared_ptr<rsf_tree_s> tree, const rsf_kernel* kernel, const double* theta,
                                 int which, double tol, const rsf_opts& o) {
  check_kernel(kernel, theta);
  RSF_CHECK((which >= RSF_SIGMA && which <= RSF_D_S2) || (which == RSF_D_L2 && kernel->anisotropic), RSF_EINVAL,
            "which must be SIGMA, D_L, D_S2 or (anisotropic kernels) D_L2");
  RSF_CHECK(tol > 0.0 && tol < 1.0, RSF_EINVAL, "tol must be in (0, 1)");
  auto h = std::make_unique<rsf_handle_s>();
  h->tree = tree;
  h->tree_raw = tree.get();
  h->opts = o;
  h->tol = tol;
  h->stream = tree->t.stream;
  RSF_CUDA(cudaGetDevice(&h->device));
  h->spd = (which == RSF_SIGMA);
  RSF_CHECK(o.precision == RSF_PREC_FP64 || o.precision == RSF_PREC_MIXED || o.precision == RSF_PREC_MIXED_DF64,
            RSF_EINVAL, "unknown precision");
  // df64 for the Cholesky-based factorization of Sigma; a derivative
  // factorization is probed at the end of factorize() and falls back to fp64
  // when df64 would cost accuracy.
  h->df = o.precision;
  h->kp.family = kernel->family;
  h->kp.alpha = kernel->alpha;
  h->kp.l = theta[0];
  h->kp.s2 = theta[1];
  h->kp.nug = theta[2];
  h->kp.which = which;
  h->kp.aniso = kernel->anisotropic;
  h->kp.l2 = kernel->anisotropic ? theta[3] : theta[0];
  int tk = prof_begin(h->stream);
  factorize(h.get());
  prof_end(tk, h->stream, PROF_FACTOR, h->flops, 0);
  check_status(h.get());
  return h.release();
}

int refine_sweeps(const rsf_handle_s* F) {
  if (!F->spd) return 0;
  // default: one sweep in the mixed forms where the residual runs in df64
  // (Matern 1/2, 3/2, 5/2; rational quadratic with integer alpha)
  if (F->opts.refine >= 0) return F->opts.refine;
  return F->opts.precision != RSF_PREC_FP64 && residual_uses_df64(F->kp) ? 1 : 0;
}

}  // namespace rsf

using namespace rsf;

#define API_BEGIN try {
#define API_END                                     \
  }                                                 \
  catch (const rsf::Exception& e) {                 \
    rsf::set_error(e.msg);                          \
    return e.code;                                  \
  }                                                 \
  catch (const std::bad_alloc&) {                   \
    rsf::set_error("host allocation failed");       \
    return RSF_ENOMEM;                              \
  }                                                 \
  catch (const std::exception& e) {                 \
    rsf::set_error(e.what());                       \
    return RSF_EINVAL;                              \
  }                                                 \
  rsf::set_error("");                               \
  return RSF_OK;

extern "C" {

void rsf_opts_default(rsf_opts* o) {
  if (!o) return;
  o->n_occ = 64;
  o->n_prox = 256;
  o->n_rings = 8;
  o->r_near = 1.0;
  o->r_in = 1.0;
  o->r_out = 2.0;
  o->oversample = 10;
  o->q0 = 64;
  o->seed = 0;
  o->precision = RSF_PREC_MIXED;
  o->trace_form = RSF_TRACE_SYM;
  o->refine = -1;
  o->probes = 64;
}

const char* rsf_last_error(void) { return g_err.c_str(); }

rsf_status rsf_selftest_wait_limit(void* stream) {
  API_BEGIN
  const int code = barrier_timeout_selftest((cudaStream_t)stream);
  RSF_CHECK(code == RSF_ETIMEOUT, RSF_ECUDA,
            "the bounded grid barrier did not report its timeout (status " + std::to_string(code) + ")");
  API_END
}

rsf_status rsf_selftest_gemm(int engine, int m, int n, int k, int ta, int tb, double alpha, const double* A,
                             int lda, const double* B, int ldb, double beta, double* C, int ldc, void* stream) {
  API_BEGIN
  RSF_CHECK(engine >= 0 && engine <= 3, RSF_EINVAL, "engine must be 0, 1, 2 or 3");
  RSF_CHECK(m >= 1 && n >= 1 && k >= 0 && A && B && C, RSF_EINVAL, "need m, n >= 1, k >= 0 and non-NULL arrays");
  RSF_CHECK(lda >= (ta ? k : m) && lda >= 1 && ldb >= (tb ? n : k) && ldb >= 1 && ldc >= m, RSF_EINVAL,
            "leading dimensions too small");
  gemm_selftest(engine, m, n, k, ta ? 1 : 0, tb ? 1 : 0, alpha, A, lda, B, ldb, beta, C, ldc, (cudaStream_t)stream);
  API_END
}

rsf_status rsf_set_allocator(rsf_alloc_fn alloc_fn, rsf_free_fn free_fn, void* ctx) {
  API_BEGIN
  RSF_CHECK((alloc_fn == nullptr) == (free_fn == nullptr), RSF_EINVAL,
            "rsf_set_allocator: alloc_fn and free_fn must both be set or both be NULL");
  std::lock_guard<std::mutex> lk(g_hook_mu);
  g_hook.alloc = alloc_fn;
  g_hook.free = free_fn;
  g_hook.ctx = alloc_fn ? ctx : nullptr;
  API_END
}

rsf_status rsf_tree_build(const double* points, int64_t n, const rsf_opts* opts, void* stream, rsf_tree* out) {
  API_BEGIN
  RSF_CHECK(points && out, RSF_EINVAL, "points and out must not be NULL");
  auto t = build_tree(points, n, resolve_opts(opts), (cudaStream_t)stream);
  std::lock_guard<std::mutex> lk(g_tree_mu);
  g_trees[t.get()] = t;
  *out = t.get();
  API_END
}

rsf_status rsf_tree_export(rsf_tree t, int64_t* n_out, int* nbox_out, int* perm, int* boxes) {
  API_BEGIN
  RSF_CHECK(t && n_out && nbox_out, RSF_EINVAL, "tree, n_out and nbox_out must not be NULL");
  const TreeData& T = t->t;
  *n_out = T.n;
  *nbox_out = (int)T.level.size();
  if (perm) {
    d2h(perm, T.perm.as<int>(), T.n, T.stream);
    sync(T.stream);
  }
  if (boxes)
    for (size_t b = 0; b < T.level.size(); b++) {
      int* r = boxes + 6 * b;
      r[0] = T.level[b]; r[1] = T.start[b]; r[2] = T.count[b];
      r[3] = T.parent[b]; r[4] = T.slot[b]; r[5] = T.box_set[b];
    }
  API_END
}

void rsf_tree_destroy(rsf_tree t) {
  if (!t) return;
  std::lock_guard<std::mutex> lk(g_tree_mu);
  g_trees.erase(t);
}

rsf_status rsf_build(const double* points, int64_t n, const rsf_kernel* kernel, const double* theta, int which,
                     double tol, const rsf_opts* opts, void* stream, rsf_handle* out) {
  API_BEGIN
  RSF_CHECK(points && out, RSF_EINVAL, "points and out must not be NULL");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  auto t = build_tree(points, n, o, (cudaStream_t)stream);
  *out = make_handle(t, kernel, theta, which, tol, o);
  API_END
}

rsf_status rsf_build_on_tree(rsf_tree tree, const rsf_kernel* kernel, const double* theta, int which, double tol,
                             const rsf_opts* opts, rsf_handle* out) {
  API_BEGIN
  RSF_CHECK(tree && out, RSF_EINVAL, "tree and out must not be NULL");
  std::shared_ptr<rsf_tree_s> t;
  {
    std::lock_guard<std::mutex> lk(g_tree_mu);
    auto it = g_trees.find(tree);
    RSF_CHECK(it != g_trees.end(), RSF_EINVAL, "unknown tree");
    t = it->second;
  }
  rsf_opts o = resolve_opts(opts);
  o.n_occ = t->opts.n_occ;
  *out = make_handle(t, kernel, theta, which, tol, o);
  API_END
}

// Per-set log-determinants (host), synchronising the stream.
static std::vector<double> logdet_sets(rsf_handle_s* h) {
  const TreeData& T = h->tree_raw->t;
  DBuf d;
  d.alloc(sizeof(double) * T.nsets, h->stream);
  LAUNCH(sum_logdet_kernel, T.nsets, 256, 0, h->stream, h->logdet_parts.as<double>(), T.box_set_d.as<int>(),
         (int)h->nboxes_total, d.as<double>(), (int64_t)1);
  std::vector<double> v(T.nsets);
  d2h(v.data(), d.as<double>(), T.nsets, h->stream);
  check_status(h);
  return v;
}

// Log-likelihood scalars of every set into sc (device, nsets x S_NSLOTS):
// alpha = F^-1 z (tree order, also returned in the caller's order when
// alpha_out is set), quad = z^T alpha, log|F|, the log-likelihood.
static void loglik_sets(rsf_handle_s* F, const double* z, double* alpha_out, DBuf& sc) {
  cudaStream_t s = F->stream;
  const TreeData& T = F->tree_raw->t;
  const int64_t n = T.n;
  const int* perm = T.perm.as<int>();
  DBuf zt, at;
  zt.alloc(sizeof(double) * n, s);
  at.alloc(sizeof(double) * n, s);
  sc.alloc(sizeof(double) * S_NSLOTS * T.nsets, s);
  sc.zero();
  LAUNCH(to_tree_kernel, cdiv(n, 256), 256, 0, s, z, n, 1, perm, n, zt.as<double>());
  solve_rows(F, RSF_OP_INV, zt.as<double>(), at.as<double>(), 1);
  // iterative refinement against the exact Sigma: alpha += F^-1 (z - Sigma alpha)
  const int sweeps = refine_sweeps(F);
  if (sweeps > 0) {
    DBuf rt, dt;
    rt.alloc(sizeof(double) * n, s);
    dt.alloc(sizeof(double) * n, s);
    for (int k = 0; k < sweeps; k++) {
      kernel_residual(F, zt.as<double>(), at.as<double>(), rt.as<double>());
      solve_rows(F, RSF_OP_INV, rt.as<double>(), dt.as<double>(), 1);
      add_into(at.as<double>(), dt.as<double>(), n, s);
    }
  }
  for (int i = 0; i < T.nsets; i++) {
    const int64_t r0 = T.set_off[i], cnt = T.set_off[i + 1] - r0;
    dot_into(zt.as<double>() + r0, at.as<double>() + r0, cnt, sc.as<double>() + (int64_t)i * S_NSLOTS + S_QUAD, s);
  }
  LAUNCH(sum_logdet_kernel, T.nsets, 256, 0, s, F->logdet_parts.as<double>(), T.box_set_d.as<int>(),
         (int)F->nboxes_total, sc.as<double>() + S_LOGDET, (int64_t)S_NSLOTS);
  LAUNCH(loglik_kernel, cdiv(T.nsets, 32), 32, 0, s, sc.as<double>(), T.set_off_d.as<int64_t>(), T.nsets);
  if (alpha_out) LAUNCH(from_tree_kernel, cdiv(n, 256), 256, 0, s, at.as<double>(), n, 1, perm, alpha_out, n);
}

// Score scalars of every set into sc (filled by loglik_sets or zeroed):
// a^T a, a^T F_l a, a^T F a per set, the peeled traces per set, the score.
// alpha_in_tree: alpha is already in tree order (else the caller's order).
static void score_sets(rsf_handle_s* F, const double* alpha, double tol_fact, double tol_peel, const rsf_opts& o,
                       DBuf& sc, bool alpha_in_tree = false) {
  cudaStream_t s = F->stream;
  const TreeData& T = F->tree_raw->t;
  const int64_t n = T.n;
  const int* perm = T.perm.as<int>();
  rsf_kernel k{F->kp.family, F->kp.alpha, F->kp.aniso};
  const double theta[4] = {F->kp.l, F->kp.s2, F->kp.nug, F->kp.l2};
  DBuf at, fl, ff;
  at.alloc(sizeof(double) * n, s);
  fl.alloc(sizeof(double) * n, s);
  ff.alloc(sizeof(double) * n, s);
  if (alpha_in_tree) RSF_CUDA(cudaMemcpyAsync(at.as<double>(), alpha, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  else LAUNCH(to_tree_kernel, cdiv(n, 256), 256, 0, s, alpha, n, 1, perm, n, at.as<double>());
  solve_rows(F, RSF_OP_APPLY, at.as<double>(), ff.as<double>(), 1);
  for (int i = 0; i < T.nsets; i++) {
    const int64_t r0 = T.set_off[i], cnt = T.set_off[i + 1] - r0;
    double* c = sc.as<double>() + (int64_t)i * S_NSLOTS;
    dot_into(at.as<double>() + r0, at.as<double>() + r0, cnt, c + S_AA, s);
    dot_into(at.as<double>() + r0, ff.as<double>() + r0, cnt, c + S_QF, s);
  }
  // one length-scale derivative at a time (l, then l2 when anisotropic), its
  // factorization freed before the next is built; Tr(F^-1) is peeled with
  // the first on shared test matrices
  const int nl = F->kp.aniso ? 2 : 1;
  for (int d = 0; d < nl; d++) {
    std::unique_ptr<rsf_handle_s> Fl(make_handle(F->tree, &k, theta, d == 0 ? RSF_D_L : RSF_D_L2, tol_fact, o));
    solve_rows(Fl.get(), RSF_OP_APPLY, at.as<double>(), fl.as<double>(), 1);
    for (int i = 0; i < T.nsets; i++) {
      const int64_t r0 = T.set_off[i], cnt = T.set_off[i + 1] - r0;
      double* c = sc.as<double>() + (int64_t)i * S_NSLOTS;
      dot_into(at.as<double>() + r0, fl.as<double>() + r0, cnt, c + (d == 0 ? S_QL : S_QL2), s);
    }
    double* const dtr[2] = {d == 0 ? sc.as<double>() + S_TNUG : nullptr, sc.as<double>() + (d == 0 ? S_TL : S_TL2)};
    peel_traces(F, Fl.get(), d == 0, tol_peel, o, dtr, (int64_t)S_NSLOTS, nullptr);
    check_status(Fl.get());
  }
  LAUNCH(score_kernel, cdiv(T.nsets, 32), 32, 0, s, sc.as<double>(), T.set_off_d.as<int64_t>(), T.nsets,
         F->kp.s2, F->kp.nug, F->kp.aniso ? 4 : 3);
}

// Profile-likelihood scalars of every set into sc (Sec. 5.5): alpha = F^-1 z
// and beta = F^-1 1 in one two-column solve (refined like gp_loglik),
// 1^T alpha, 1^T beta, gamma = (Sigma + 1 1^T)^-1 z (tree order, into gt),
// z^T gamma and log|F|; profile_kernel then forms the profile log-likelihood.
static void profile_sets(rsf_handle_s* F, const double* z, DBuf& gt, DBuf& sc) {
  cudaStream_t s = F->stream;
  const TreeData& T = F->tree_raw->t;
  const int64_t n = T.n;
  const int* perm = T.perm.as<int>();
  // x = [z | 1] and y = [alpha | beta] as tree-order columns; P, Q hold the
  // row-major n x 2 blocks the solves take
  DBuf X, Y, P, Q;
  X.alloc(sizeof(double) * 2 * n, s);
  Y.alloc(sizeof(double) * 2 * n, s);
  P.alloc(sizeof(double) * 2 * n, s);
  Q.alloc(sizeof(double) * 2 * n, s);
  gt.alloc(sizeof(double) * n, s);
  sc.alloc(sizeof(double) * S_NSLOTS * T.nsets, s);
  sc.zero();
  double* x = X.as<double>();
  double* y = Y.as<double>();
  const int nb = (int)cdiv(n, 256);
  LAUNCH(to_tree_kernel, nb, 256, 0, s, z, n, 1, perm, n, x);
  LAUNCH(fill_kernel, nb, 256, 0, s, x + n, n, 1.0);
  LAUNCH(pack2_kernel, nb, 256, 0, s, x, x + n, n, P.as<double>());
  solve_rows(F, RSF_OP_INV, P.as<double>(), Q.as<double>(), 2);
  LAUNCH(unpack2_kernel, nb, 256, 0, s, Q.as<double>(), n, y, y + n);
  const int sweeps = refine_sweeps(F);
  if (sweeps > 0) {
    DBuf R;
    R.alloc(sizeof(double) * 2 * n, s);
    double* r = R.as<double>();
    for (int k = 0; k < sweeps; k++) {
      for (int c = 0; c < 2; c++) kernel_residual(F, x + c * n, y + c * n, r + c * n);
      LAUNCH(pack2_kernel, nb, 256, 0, s, r, r + n, n, P.as<double>());
      solve_rows(F, RSF_OP_INV, P.as<double>(), Q.as<double>(), 2);
      LAUNCH(unpack2_kernel, nb, 256, 0, s, Q.as<double>(), n, r, r + n);
      add_into(y, r, 2 * n, s);
    }
  }
  for (int i = 0; i < T.nsets; i++) {
    const int64_t r0 = T.set_off[i], cnt = T.set_off[i + 1] - r0;
    double* c = sc.as<double>() + (int64_t)i * S_NSLOTS;
    dot_into(x + n + r0, y + r0, cnt, c + S_ONEA, s);
    dot_into(x + n + r0, y + n + r0, cnt, c + S_ONEB, s);
    dot_into(x + r0, y + r0, cnt, c + S_QUAD, s);
  }
  LAUNCH(profile_gamma_kernel, nb, 256, 0, s, y, y + n, n, T.set_off_d.as<int64_t>(), T.nsets, sc.as<double>(),
         gt.as<double>());
  for (int i = 0; i < T.nsets; i++) {
    const int64_t r0 = T.set_off[i], cnt = T.set_off[i + 1] - r0;
    dot_into(x + r0, gt.as<double>() + r0, cnt, sc.as<double>() + (int64_t)i * S_NSLOTS + S_PQ, s);
  }
  LAUNCH(sum_logdet_kernel, T.nsets, 256, 0, s, F->logdet_parts.as<double>(), T.box_set_d.as<int>(),
         (int)F->nboxes_total, sc.as<double>() + S_LOGDET, (int64_t)S_NSLOTS);
}

// In-place operator on caller-order columns B (n x nrhs, leading dimension ldb).
static void solve_caller(rsf_handle_s* h, int op, double* B, int64_t ldb, int nrhs) {
  cudaStream_t s = h->stream;
  const int64_t n = h->tree_raw->t.n;
  const int* perm = h->tree_raw->t.perm.as<int>();
  DBuf X, Y;
  X.alloc(sizeof(double) * n * nrhs, s);
  Y.alloc(sizeof(double) * n * nrhs, s);
  LAUNCH(to_tree_kernel, cdiv(n * nrhs, 256), 256, 0, s, B, ldb, nrhs, perm, n, X.as<double>());
  solve_rows(h, op, X.as<double>(), Y.as<double>(), nrhs);
  LAUNCH(from_tree_kernel, cdiv(n * nrhs, 256), 256, 0, s, Y.as<double>(), n, nrhs, perm, B, ldb);
}

rsf_status rsf_logdet(rsf_handle h, double* out) {
  API_BEGIN
  RSF_CHECK(h && out, RSF_EINVAL, "handle and out must not be NULL");
  RSF_CHECK(h->spd, RSF_EINVAL, "log-determinant of a derivative factorization is not defined here");
  std::vector<double> v = logdet_sets(h);
  double t = 0.0;
  for (double x : v) t += x;
  *out = t;
  API_END
}

rsf_status rsf_logdet_sets(rsf_handle h, double* out) {
  API_BEGIN
  RSF_CHECK(h && out, RSF_EINVAL, "handle and out must not be NULL");
  RSF_CHECK(h->spd, RSF_EINVAL, "log-determinant of a derivative factorization is not defined here");
  std::vector<double> v = logdet_sets(h);
  for (size_t i = 0; i < v.size(); i++) out[i] = v[i];
  API_END
}

rsf_status rsf_solve(rsf_handle h, double* B, int64_t ldb, int nrhs, int op) {
  API_BEGIN
  RSF_CHECK(h && B, RSF_EINVAL, "handle and B must not be NULL");
  const int64_t n = h->tree_raw->t.n;
  RSF_CHECK(nrhs >= 1 && ldb >= n, RSF_EINVAL, "need nrhs >= 1 and ldb >= n");
  RSF_CHECK(op >= RSF_OP_INV && op <= RSF_OP_INV_SQRT_T, RSF_EINVAL, "unknown op");
  RSF_CHECK(h->spd || op == RSF_OP_APPLY, RSF_EINVAL, "only APPLY is defined for a derivative factorization");
  solve_caller(h, op, B, ldb, nrhs);
  API_END
}

rsf_status rsf_solve_noalloc(rsf_handle h, double* B, int64_t ldb, int nrhs, int op) {
  API_BEGIN
  RSF_CHECK(h && B, RSF_EINVAL, "handle and B must not be NULL");
  const int64_t n = h->tree_raw->t.n;
  RSF_CHECK(nrhs >= 1 && ldb >= n, RSF_EINVAL, "need nrhs >= 1 and ldb >= n");
  RSF_CHECK(op >= RSF_OP_INV && op <= RSF_OP_INV_SQRT_T, RSF_EINVAL, "unknown op");
  RSF_CHECK(h->spd || op == RSF_OP_APPLY, RSF_EINVAL, "only APPLY is defined for a derivative factorization");
  solve_noalloc(h, B, ldb, nrhs, op);
  API_END
}

rsf_status rsf_peel_trace(rsf_handle F, rsf_handle Fk, double tol_peel, const rsf_opts* opts, double* trace) {
  API_BEGIN
  RSF_CHECK(F && trace, RSF_EINVAL, "F and trace must not be NULL");
  RSF_CHECK(F->spd, RSF_EINVAL, "F must factor Sigma");
  RSF_CHECK(!Fk || same_tree(Fk->tree_raw, F->tree_raw), RSF_EINVAL, "F and Fk must be built on the same tree");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  double* const dnone[2] = {nullptr, nullptr};
  const int nsets = F->tree_raw->t.nsets;
  std::vector<double> t(2 * nsets, 0.0);
  peel_traces(F, Fk, false, tol_peel, o, dnone, 0, t.data());
  check_status(F);
  if (Fk) check_status(Fk);
  double tot = 0.0;
  for (int i = 0; i < nsets; i++) tot += t[(Fk ? 1 : 0) * nsets + i];
  *trace = tot;
  API_END
}

rsf_status gp_loglik(rsf_handle F, const double* z, double* alpha_out, double* loglik, double* quad) {
  API_BEGIN
  RSF_CHECK(F && z && loglik, RSF_EINVAL, "F, z and loglik must not be NULL");
  RSF_CHECK(F->spd, RSF_EINVAL, "F must factor Sigma");
  const int nsets = F->tree_raw->t.nsets;
  DBuf sc;
  loglik_sets(F, z, alpha_out, sc);
  std::vector<double> h((size_t)S_NSLOTS * nsets);
  d2h(h.data(), sc.as<double>(), h.size(), F->stream);
  check_status(F);
  double ll = 0.0, q = 0.0;
  for (int i = 0; i < nsets; i++) {
    ll += h[(size_t)i * S_NSLOTS + S_LOGLIK];
    q += h[(size_t)i * S_NSLOTS + S_QUAD];
  }
  *loglik = ll;
  if (quad) *quad = q;
  API_END
}

rsf_status gp_score(rsf_handle F, const double* alpha, double tol_fact, double tol_peel, const rsf_opts* opts,
                    double* score, double* terms) {
  API_BEGIN
  RSF_CHECK(F && alpha && score, RSF_EINVAL, "F, alpha and score must not be NULL");
  RSF_CHECK(F->spd, RSF_EINVAL, "F must factor Sigma");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  const int nsets = F->tree_raw->t.nsets;
  DBuf sc;
  sc.alloc(sizeof(double) * S_NSLOTS * nsets, F->stream);
  sc.zero();
  score_sets(F, alpha, tol_fact, tol_peel, o, sc);
  std::vector<double> h((size_t)S_NSLOTS * nsets);
  d2h(h.data(), sc.as<double>(), h.size(), F->stream);
  check_status(F);
  const int p = F->kp.aniso ? 4 : 3;
  for (int i = 0; i < p; i++) {
    score[i] = 0.0;
    for (int j = 0; j < nsets; j++) score[i] += h[(size_t)j * S_NSLOTS + S_G0 + i];
  }
  if (terms)
    for (int i = 0; i < p; i++) {
      terms[i] = terms[p + i] = 0.0;
      for (int j = 0; j < nsets; j++) {
        terms[i] += h[(size_t)j * S_NSLOTS + S_Q0 + i];
        terms[p + i] += h[(size_t)j * S_NSLOTS + S_R0 + i];
      }
    }
  API_END
}

// Algorithm 1 on a forest: per-set log-likelihoods and (score != NULL) scores.
static void loglik_and_score_forest(std::shared_ptr<rsf_tree_s> t, const double* z, const rsf_kernel* kernel,
                                    const double* theta, double tol_fact, double tol_peel, const rsf_opts& o,
                                    double* loglik, double* score, double* terms) {
  const TreeData& T = t->t;
  cudaStream_t s = T.stream;
  std::unique_ptr<rsf_handle_s> F(make_handle(t, kernel, theta, RSF_SIGMA, tol_fact, o));
  DBuf alpha, sc;
  alpha.alloc(sizeof(double) * T.n, s);
  loglik_sets(F.get(), z, alpha.as<double>(), sc);
  if (score) score_sets(F.get(), alpha.as<double>(), tol_fact, tol_peel, o, sc);
  std::vector<double> h((size_t)S_NSLOTS * T.nsets);
  d2h(h.data(), sc.as<double>(), h.size(), s);
  check_status(F.get());
  const int p = nparams(kernel);
  for (int i = 0; i < T.nsets; i++) {
    const double* c = h.data() + (size_t)i * S_NSLOTS;
    loglik[i] = c[S_LOGLIK];
    if (score)
      for (int j = 0; j < p; j++) score[p * i + j] = c[S_G0 + j];
    if (score && terms)
      for (int j = 0; j < p; j++) {
        terms[2 * p * i + j] = c[S_Q0 + j];
        terms[2 * p * i + p + j] = c[S_R0 + j];
      }
  }
}

rsf_status gp_loglik_and_score(const double* points, const double* z, int64_t n, const rsf_kernel* kernel,
                               const double* theta, double tol_fact, double tol_peel, const rsf_opts* opts,
                               void* stream, double* loglik, double* score, double* terms) {
  API_BEGIN
  RSF_CHECK(points && z && loglik, RSF_EINVAL, "points, z and loglik must not be NULL");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  auto t = build_tree(points, n, o, (cudaStream_t)stream);
  loglik_and_score_forest(t, z, kernel, theta, tol_fact, tol_peel, o, loglik, score, terms);
  API_END
}

static std::vector<int64_t> set_offsets(int nsets, const int64_t* offsets) {
  RSF_CHECK(nsets >= 1 && offsets != nullptr, RSF_EINVAL, "need nsets >= 1 and an offsets array");
  return std::vector<int64_t>(offsets, offsets + nsets + 1);
}

rsf_status rsf_build_batched(int nsets, const int64_t* offsets, const double* points, const rsf_kernel* kernel,
                             const double* theta, int which, double tol, const rsf_opts* opts, void* stream,
                             rsf_handle* out) {
  API_BEGIN
  RSF_CHECK(points && out, RSF_EINVAL, "points and out must not be NULL");
  rsf_opts o = resolve_opts(opts);
  auto t = build_forest(points, set_offsets(nsets, offsets), o, (cudaStream_t)stream);
  *out = make_handle(t, kernel, theta, which, tol, o);
  API_END
}

rsf_status gp_loglik_and_score_batched(int nsets, const int64_t* offsets, const double* points, const double* z,
                                       const rsf_kernel* kernel, const double* theta, double tol_fact,
                                       double tol_peel, const rsf_opts* opts, void* stream, double* loglik,
                                       double* score, double* terms) {
  API_BEGIN
  RSF_CHECK(points && z && loglik, RSF_EINVAL, "points, z and loglik must not be NULL");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  auto t = build_forest(points, set_offsets(nsets, offsets), o, (cudaStream_t)stream);
  loglik_and_score_forest(t, z, kernel, theta, tol_fact, tol_peel, o, loglik, score, terms);
  API_END
}

// Profile likelihood (Sec. 5.5) on a forest: per-set lt and (score != NULL)
// its gradient; terms per set (2p + 4): gamma^T Sigma_k gamma (p), the traces
// (p), z^T gamma, log|F|, 1^T Sigma^-1 z, 1^T Sigma^-1 1.
static void profile_forest(std::shared_ptr<rsf_tree_s> t, const double* z, const rsf_kernel* kernel,
                           const double* theta, double tol_fact, double tol_peel, const rsf_opts& o, double* loglik,
                           double* score, double* terms) {
  const TreeData& T = t->t;
  cudaStream_t s = T.stream;
  std::unique_ptr<rsf_handle_s> F(make_handle(t, kernel, theta, RSF_SIGMA, tol_fact, o));
  DBuf gt, sc;
  profile_sets(F.get(), z, gt, sc);
  if (score) score_sets(F.get(), gt.as<double>(), tol_fact, tol_peel, o, sc, true);
  LAUNCH(profile_kernel, cdiv(T.nsets, 32), 32, 0, s, sc.as<double>(), T.set_off_d.as<int64_t>(), T.nsets,
         score ? 1 : 0, nparams(kernel));
  std::vector<double> h((size_t)S_NSLOTS * T.nsets);
  d2h(h.data(), sc.as<double>(), h.size(), s);
  check_status(F.get());
  const int p = nparams(kernel);
  for (int i = 0; i < T.nsets; i++) {
    const double* c = h.data() + (size_t)i * S_NSLOTS;
    loglik[i] = c[S_LOGLIK];
    if (score)
      for (int j = 0; j < p; j++) score[p * i + j] = c[S_G0 + j];
    if (terms) {
      double* tr = terms + (2 * p + 4) * i;
      for (int j = 0; j < p; j++) {
        tr[j] = score ? c[S_Q0 + j] : 0.0;
        tr[p + j] = score ? c[S_R0 + j] : 0.0;
      }
      tr[2 * p] = c[S_PQ];
      tr[2 * p + 1] = c[S_LOGDET];
      tr[2 * p + 2] = c[S_ONEA];
      tr[2 * p + 3] = c[S_ONEB];
    }
  }
}

rsf_status gp_profile_loglik_and_score(const double* points, const double* z, int64_t n, const rsf_kernel* kernel,
                                       const double* theta, double tol_fact, double tol_peel, const rsf_opts* opts,
                                       void* stream, double* loglik, double* score, double* terms) {
  API_BEGIN
  RSF_CHECK(points && z && loglik, RSF_EINVAL, "points, z and loglik must not be NULL");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  auto t = build_tree(points, n, o, (cudaStream_t)stream);
  profile_forest(t, z, kernel, theta, tol_fact, tol_peel, o, loglik, score, terms);
  API_END
}

rsf_status gp_profile_loglik_and_score_batched(int nsets, const int64_t* offsets, const double* points,
                                               const double* z, const rsf_kernel* kernel, const double* theta,
                                               double tol_fact, double tol_peel, const rsf_opts* opts, void* stream,
                                               double* loglik, double* score, double* terms) {
  API_BEGIN
  RSF_CHECK(points && z && loglik, RSF_EINVAL, "points, z and loglik must not be NULL");
  RSF_CHECK(tol_peel > 0.0 && tol_peel < 1.0, RSF_EINVAL, "tol_peel must be in (0, 1)");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  auto t = build_forest(points, set_offsets(nsets, offsets), o, (cudaStream_t)stream);
  profile_forest(t, z, kernel, theta, tol_fact, tol_peel, o, loglik, score, terms);
  API_END
}

rsf_status gp_conditional(const double* points, int64_t n, const double* z, const double* new_points, int64_t m,
                          const rsf_kernel* kernel, const double* theta, double tol, const rsf_opts* opts,
                          void* stream, int method, double* mean, const double* w, int q, double* samples) {
  API_BEGIN
  RSF_CHECK(points && z && new_points && mean, RSF_EINVAL, "points, z, new_points and mean must not be NULL");
  RSF_CHECK(n >= 1 && m >= 1, RSF_EINVAL, "need n >= 1 observed and m >= 1 new points");
  RSF_CHECK(method == RSF_COND_RSF || method == RSF_COND_DIRECT, RSF_EINVAL, "unknown method");
  RSF_CHECK(q >= 0, RSF_EINVAL, "q must be >= 0");
  RSF_CHECK(q == 0 || (w && samples && method == RSF_COND_RSF), RSF_EINVAL,
            "samples need w, samples and method RSF_COND_RSF");
  rsf_opts o = resolve_opts(opts);
  check_kernel(kernel, theta);
  cudaStream_t s = (cudaStream_t)stream;
  auto t2 = build_tree(points, n, o, s);
  std::unique_ptr<rsf_handle_s> F2(make_handle(t2, kernel, theta, RSF_SIGMA, tol, o));
  // alpha = Sigma_22^-1 z (caller order), refined like gp_loglik
  DBuf a, sc;
  a.alloc(sizeof(double) * n, s);
  loglik_sets(F2.get(), z, a.as<double>(), sc);
  if (method == RSF_COND_DIRECT) {
    cross_matvec(F2->kp, points, a.as<double>(), n, new_points, m, mean, s);
  } else {
    // the joint matrix of [new points; points]; Sigma_12 v = (F [0; v])(0:m)
    const int64_t nj = n + m;
    DBuf J;
    J.alloc(sizeof(double) * 2 * nj, s);
    RSF_CUDA(cudaMemcpyAsync(J.as<double>(), new_points, sizeof(double) * 2 * m, cudaMemcpyDeviceToDevice, s));
    RSF_CUDA(cudaMemcpyAsync(J.as<double>() + 2 * m, points, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    auto tj = build_tree(J.as<double>(), nj, o, s);
    std::unique_ptr<rsf_handle_s> FJ(make_handle(tj, kernel, theta, RSF_SIGMA, tol, o));
    DBuf V;
    V.alloc(sizeof(double) * nj, s);
    RSF_CUDA(cudaMemsetAsync(V.as<double>(), 0, sizeof(double) * m, s));
    RSF_CUDA(cudaMemcpyAsync(V.as<double>() + m, a.as<double>(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    solve_caller(FJ.get(), RSF_OP_APPLY, V.as<double>(), nj, 1);
    RSF_CUDA(cudaMemcpyAsync(mean, V.as<double>(), sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    if (q > 0) {
      // y = F^1/2 w; samples = mean + y_1 - Sigma_12 Sigma_22^-1 y_2
      DBuf Y, Z, P;
      Y.alloc(sizeof(double) * nj * q, s);
      Z.alloc(sizeof(double) * n * q, s);
      P.alloc(sizeof(double) * nj * q, s);
      RSF_CUDA(cudaMemcpyAsync(Y.as<double>(), w, sizeof(double) * nj * q, cudaMemcpyDeviceToDevice, s));
      solve_caller(FJ.get(), RSF_OP_SQRT, Y.as<double>(), nj, q);
      RSF_CUDA(cudaMemcpy2DAsync(Z.as<double>(), sizeof(double) * n, Y.as<double>() + m, sizeof(double) * nj,
                                 sizeof(double) * n, q, cudaMemcpyDeviceToDevice, s));
      solve_caller(F2.get(), RSF_OP_INV, Z.as<double>(), n, q);
      RSF_CUDA(cudaMemsetAsync(P.as<double>(), 0, sizeof(double) * nj * q, s));
      RSF_CUDA(cudaMemcpy2DAsync(P.as<double>() + m, sizeof(double) * nj, Z.as<double>(), sizeof(double) * n,
                                 sizeof(double) * n, q, cudaMemcpyDeviceToDevice, s));
      solve_caller(FJ.get(), RSF_OP_APPLY, P.as<double>(), nj, q);
      LAUNCH(cond_combine_kernel, cdiv(m * q, 256), 256, 0, s, mean, Y.as<double>(), nj, P.as<double>(), nj, m, q,
             samples, m);
    }
    check_status(FJ.get());
  }
  check_status(F2.get());
  API_END
}

rsf_status rsf_get_info(rsf_handle h, rsf_info_t* info) {
  API_BEGIN
  RSF_CHECK(h && info, RSF_EINVAL, "handle and info must not be NULL");
  info->n = h->tree_raw->t.n;
  info->levels = (int)h->levels.size();
  int64_t nb = 0;
  for (auto& l : h->levels) nb += l.nb;
  info->boxes = nb;
  info->root_size = h->levels.empty() ? 0 : (int)h->levels[0].nrows;
  info->max_rank = h->max_rank;
  info->max_active = h->max_active;
  info->factor_entries = h->factor_entries;
  info->flops = h->flops;
  info->kernel_evals = h->kevals;
  info->nsets = h->tree_raw->t.nsets;
  info->solve_df64 = h->df;
  info->probe_rel_diff = h->probe_rel_diff;
  API_END
}

void rsf_profile_enable(int on) {
  if (!on) prof_drain();
  g_prof_on = on != 0;
}

rsf_status rsf_profile_read(int category, int reset, int64_t* launches, double* ms, double* flops, double* bytes) {
  API_BEGIN
  RSF_CHECK(category >= 0 && category < PROF_NCAT, RSF_EINVAL, "unknown profile category");
  prof_drain();
  ProfAcc& a = g_prof_acc[category];
  if (launches) *launches = a.launches;
  if (ms) *ms = a.ms;
  if (flops) *flops = a.flops;
  if (bytes) *bytes = a.bytes;
  if (reset) a = ProfAcc{};
  API_END
}

int64_t rsf_launch_count(int reset) {
  int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

void rsf_destroy(rsf_handle h) {
  if (!h) return;
  cudaStream_t s = h->stream;
  delete h;
  cudaStreamSynchronize(s);
}

}  // extern "C"
