// Batched ragged fp64 dense kernels: see dense.cuh.
#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "dense.cuh"
#include "df64.cuh"

namespace rsf {

// ===================================================================== GEMM
// Tile BM x BN (64 x 32), BK = 16; each thread owns an RM x RN (4 x 4)
// register tile (rows tm + TM i, cols tn + TN j with TM = BM / RM,
// TN = BN / RN), so a CTA has TM x TN (128) threads.
#ifndef GEMM_BM
#define GEMM_BM 64
#endif
#ifndef GEMM_BN
#define GEMM_BN 32
#endif
#ifndef GEMM_BK
#define GEMM_BK 16
#endif
// Four resident CTAs per SM (registers capped at 128) and a k loop unrolled
// by two: measured on GB300 against full unrolling with two CTAs per SM,
// 2.4x on 40 x 40 leaf blocks and 1.3x on 1000 x 1000 blocks in df64.  A
// 128 x 32 tile with 8 x 4 per thread and BK = 8 is 5-11 % faster on
// isolated leaf and mid-level shapes but 8 % slower across a whole
// evaluation (more M-tile waste on the narrow column blocks of the peeling).
#ifndef GEMM_MIN_BLOCKS
#define GEMM_MIN_BLOCKS 4
#endif
#ifndef GEMM_KUNROLL
#define GEMM_KUNROLL 2
#endif
constexpr int BM = GEMM_BM, BN = GEMM_BN, BK = GEMM_BK;
#ifndef GEMM_RM
#define GEMM_RM 4
#endif
constexpr int RM = GEMM_RM, RN = 4;   // register tile of a thread: RM x RN
constexpr int TM = BM / RM, TN = BN / RN, GT = TM * TN, KUNROLL = GEMM_KUNROLL;
static_assert((BM * BK) % GT == 0 && (BN * BK) % GT == 0, "tile loads must split evenly");


// Asynchronous 8-byte global -> shared copy (zero-fill when !pred).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  int sz = pred ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Element access for the two arithmetic modes: fp64, or df64 (8-byte
// float2 pairs, products accumulated with error-free transformations).
template <bool DF> struct Arith;
template <> struct Arith<false> {
  typedef double T;
  typedef double Acc;
  static __device__ __forceinline__ T load(const double* p) { return *p; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ Acc acc0() { return 0.0; }
  static __device__ __forceinline__ void mac(Acc& c, T a, T b) { c = fma(a, b, c); }
  static __device__ __forceinline__ void store(double* p, Acc c, double alpha, double beta) {
    double v = alpha * c;
    if (beta != 0.0) v = fma(beta, *p, v);
    *p = v;
  }
};
template <> struct Arith<true> {
  typedef df64 T;
  typedef dfacc Acc;
  static __device__ __forceinline__ T load(const double* p) {
    float2 f = *reinterpret_cast<const float2*>(p);
    return {f.x, f.y};
  }
  static __device__ __forceinline__ T zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ Acc acc0() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void mac(Acc& c, T a, T b) { df_mac(c, a, b); }
  static __device__ __forceinline__ void store(double* p, Acc c, double alpha, double beta) {
    df64 v = df_scale(df_of_acc(c), (float)alpha);
    if (beta != 0.0) {
      float2 o = *reinterpret_cast<const float2*>(p);
      df64 old = {o.x, o.y};
      if (beta != 1.0) old = df_scale(old, (float)beta);
      v = df_add(v, old);
    }
    *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo);
  }
};

template <bool DF>
__global__ void __launch_bounds__(GT, GEMM_MIN_BLOCKS) gemm_kernel(const GemmDesc* __restrict__ descs,
                                                  const int* __restrict__ prefix, int nprob,
                                                  GemmBases bases) {
  typedef Arith<DF> AR;
  typedef typename AR::T T;
  const int p = find_prob(prefix, nprob, blockIdx.x);
  const GemmDesc d = descs[p];
  const int M = d.M >= 0 ? d.M : bases.M;
  const int N = d.N, K = d.K;
  const int n0 = (blockIdx.x - prefix[p]) * BN;
  const int m0 = blockIdx.y * BM;
  if (m0 >= M || n0 >= N) return;
  if (d.lowC && n0 > m0 + BM - 1) return;
  const int lda = d.lda >= 0 ? d.lda : bases.ld;
  const int ldb = d.ldb >= 0 ? d.ldb : bases.ld;
  const int ldc = d.ldc >= 0 ? d.ldc : bases.ld;
  const double* pa = d.abase == 0 ? bases.p[0] : d.abase == 1 ? bases.p[1] : d.abase == 2 ? bases.p[2] : bases.p[3];
  const double* pb = d.bbase == 0 ? bases.p[0] : d.bbase == 1 ? bases.p[1] : d.bbase == 2 ? bases.p[2] : bases.p[3];
  double* pc = d.cbase == 0 ? bases.p[0] : d.cbase == 1 ? bases.p[1] : d.cbase == 2 ? bases.p[2] : bases.p[3];
  const int64_t sa = d.abase == 0 ? bases.sc[0] : d.abase == 1 ? bases.sc[1] : d.abase == 2 ? bases.sc[2] : bases.sc[3];
  const int64_t sb = d.bbase == 0 ? bases.sc[0] : d.bbase == 1 ? bases.sc[1] : d.bbase == 2 ? bases.sc[2] : bases.sc[3];
  const int64_t scc = d.cbase == 0 ? bases.sc[0] : d.cbase == 1 ? bases.sc[1] : d.cbase == 2 ? bases.sc[2] : bases.sc[3];
  const double* __restrict__ A = pa + d.a * sa + d.m0;
  const double* __restrict__ B = pb + d.b * sb;
  double* __restrict__ C = pc + d.c * scc + d.m0;
  int k0 = 0, k1 = K;
  if (d.triB == 1) k0 = min(n0, K);
  if (d.triB == 2) k1 = min(K, n0 + BN);

  // Two shared-memory stages filled with cp.async: the loads of tile k+1 are
  // in flight while tile k is multiplied.  Out-of-range and masked elements
  // are zero-filled by the copy itself (source size 0).
  __shared__ __align__(16) T sA[2][BK][BM + 1];
  __shared__ __align__(16) T sB[2][BK][BN + 1];
  const int t = threadIdx.x;
  const int tm = t % TM, tn = t / TM;
  typename AR::Acc acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; i++)
#pragma unroll
    for (int j = 0; j < RN; j++) acc[i][j] = AR::acc0();

  auto load_tile = [&](int kb, int st) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / GT; r++) {
      int idx = t + r * GT;
      int mm, kk;
      if (!d.ta) { mm = idx % BM; kk = idx / BM; } else { kk = idx % BK; mm = idx / BK; }
      int gm = m0 + mm, gk = kb + kk;
      bool ok = gm < M && gk < k1;
      const double* src = A;
      if (ok) {
        if (d.gatherK) src = A + gm + (int64_t)bases.kidx[d.kofs + gk] * lda;
        else src = d.ta ? A + gk + (int64_t)gm * lda : A + gm + (int64_t)gk * lda;
      }
      cp_async8(&sA[st][kk][mm], src, ok);
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / GT; r++) {
      int idx = t + r * GT;
      int nn, kk;
      if (!d.tb) { kk = idx % BK; nn = idx / BK; } else { nn = idx % BN; kk = idx / BN; }
      int gn = n0 + nn, gk = kb + kk;
      bool ok = gn < N && gk < k1;
      if (ok && !d.gatherK && !d.gatherN) ok = !((d.triB == 1 && gk < gn) || (d.triB == 2 && gk > gn));
      const double* src = B;
      if (ok) {
        if (d.gatherK) src = B + (bases.kidx[d.kofs + gk] - d.kb0) + (int64_t)gn * ldb;
        else if (d.gatherN) src = B + (bases.kidx[d.nofs + gn] - d.nb0) + (int64_t)gk * ldb;
        else src = d.tb ? B + gn + (int64_t)gk * ldb : B + gk + (int64_t)gn * ldb;
      }
      cp_async8(&sB[st][kk][nn], src, ok);
    }
    cp_async_commit();
  };

  int st = 0;
  if (k0 < k1) load_tile(k0, 0);
  for (int kb = k0; kb < k1; kb += BK) {
    const bool more = kb + BK < k1;
    if (more) load_tile(kb + BK, st ^ 1);
    if (more) cp_async_wait<1>(); else cp_async_wait<0>();
    __syncthreads();
#pragma unroll KUNROLL
    for (int kk = 0; kk < BK; kk++) {
      T a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; i++) a[i] = sA[st][kk][tm + TM * i];
#pragma unroll
      for (int j = 0; j < RN; j++) b[j] = sB[st][kk][tn + TN * j];
#pragma unroll
      for (int i = 0; i < RM; i++)
#pragma unroll
        for (int j = 0; j < RN; j++) AR::mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
    st ^= 1;
  }
  const double alpha = d.alpha * bases.alpha_scale, beta = d.beta;
#pragma unroll
  for (int i = 0; i < RM; i++) {
    int gm = m0 + tm + TM * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < RN; j++) {
      int gn = n0 + tn + TN * j;
      if (gn >= N) continue;
      if (d.lowC && gm < gn) continue;
      const int64_t cn = d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn;
      AR::store(C + gm + cn * ldc, acc[i][j], alpha, beta);
    }
  }
}

void GemmBatch::build(const std::vector<GemmDesc>& d, cudaStream_t s) {
  nprob = (int)d.size();
  std::vector<int> pre(nprob + 1, 0);
  std::vector<int2> nttc;
  maxM = 0;
  anyLaunchM = false;
  fixedMNK = launchNK = fixedBytes = launchBytesPerM = launchBytes0 = 0;
  for (int i = 0; i < nprob; i++) {
    pre[i + 1] = pre[i] + std::max(0, cdiv(d[i].N, BN));
    for (int c = 0; c < d[i].N; c += TC_BN) nttc.push_back(make_int2(i, c));
    if (d[i].M < 0) anyLaunchM = true; else maxM = std::max(maxM, d[i].M);
    // nonzero (k, n) pairs of op(B) and the computed part of C
    double N = d[i].N, K = d[i].K, nk;
    if (d[i].triB == 1) {          // op(B)[k, n] != 0 for k >= n
      double m = std::min(N, K);
      nk = m * K - m * (m - 1) / 2;
    } else if (d[i].triB == 2) {   // op(B)[k, n] != 0 for k <= n
      double m = std::min(N, K);
      nk = m * (m + 1) / 2 + (N - m) * K;
    } else {
      nk = N * K;
    }
    double cfrac = d[i].lowC ? 0.5 * (1.0 + 1.0 / std::max(1.0, N)) : 1.0;
    if (d[i].M < 0) {
      launchNK += nk * cfrac;
      launchBytesPerM += 8.0 * (K + 2.0 * N * cfrac);
      launchBytes0 += 8.0 * nk;
    } else {
      fixedMNK += (double)d[i].M * nk * cfrac;
      fixedBytes += 8.0 * ((double)d[i].M * K + nk + 2.0 * d[i].M * N * cfrac);
    }
  }
  ntilesN = pre[nprob];
  ntilesN_tc = (int)nttc.size();
  upload(desc, d, s);
  upload(prefix, pre, s);
  upload(ntile_tc, nttc, s);
  // plan of the pre-sliced tensor-core engine
  std::vector<TcDescPlan> dp(nprob);
  std::vector<TcEntryPlan> ep(nttc.size());
  tc_pi = tc_qi = tc_pa = tc_qa = tc_pe = tc_qe = tc_bblk = tc_be = tc_pib = 0;
  for (int i = 0; i < nprob; i++) {
    const int K = std::max(0, d[i].K);
    TcDescPlan& q = dp[i];
    q.nch = cdiv(K, TC_KC);
    q.nsb = cdiv(K, TC_SBK);
    q.pi = tc_pi; q.qi = tc_qi; q.pa = tc_pa; q.qa = tc_qa; q.pe = tc_pe; q.qe = tc_qe;
    if (d[i].M >= 0) {
      const int64_t mt = cdiv(d[i].M, TC_BM);
      tc_pi += mt * q.nsb;
      tc_pa += mt * q.nch;
      tc_pe += mt * TC_BM * q.nsb;
    } else {
      tc_qi += q.nsb;
      tc_qa += q.nch;
      tc_qe += (int64_t)TC_BM * q.nsb;
    }
  }
  for (size_t e = 0; e < nttc.size(); e++) {
    const TcDescPlan& q = dp[nttc[e].x];
    ep[e] = TcEntryPlan{tc_bblk, tc_be, tc_pib};
    tc_bblk += q.nch;
    tc_be += (int64_t)TC_BN * q.nsb;
    tc_pib += q.nsb;
  }
  tc_dplan_h = std::move(dp);
  tc_eplan_h = std::move(ep);
  tc_dplan.release();
  tc_eplan.release();
}

void GemmBatch::run(const GemmBases& b, cudaStream_t s) const {
  if (nprob == 0 || ntilesN == 0) return;
  int M = maxM;
  if (anyLaunchM) M = std::max(M, b.M);
  if (M <= 0) return;
  dim3 grid(ntilesN, cdiv(M, BM));
  RSF_CHECK(grid.y <= 65535, RSF_EINVAL, "gemm: M too large");
  int tok = prof_begin(s);
  const bool tensor = (b.df == 1 || b.df == 3) && M >= TC_MIN_M;
  if (tensor && b.df == 1)
    tc_gemm_pre_run(*this, b, M, s);
  else if (tensor)
    tc_gemm_run(*this, b, M, s);
  else if (b.df)
    LAUNCH(gemm_kernel<true>, grid, GT, 0, s, desc.as<GemmDesc>(), prefix.as<int>(), nprob, b);
  else
    LAUNCH(gemm_kernel<false>, grid, GT, 0, s, desc.as<GemmDesc>(), prefix.as<int>(), nprob, b);
  if (tok >= 0) {
    double Ml = anyLaunchM ? (double)b.M : 0.0;
    prof_end(tok, s, tensor ? PROF_GEMM_TC : b.df ? PROF_GEMM_DF : PROF_GEMM, 2.0 * (fixedMNK + Ml * launchNK),
             fixedBytes + (anyLaunchM ? launchBytes0 + Ml * launchBytesPerM : 0.0));
  }
}

// ============================================================ pivoted QR
constexpr int QR_THREADS = 256;
constexpr long long QR_BARRIER_SPINS = 1ll << 25;   // x ~64 ns sleeps: a few seconds
constexpr double QR_TOL3Z = 1.4901161193847656e-08;  // sqrt(2^-52)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long pivot_key(double norm2, int col) {
  // Non-negative doubles order like their bit patterns; the low 16 bits carry
  // the complement of the column so that ties go to the lowest column.
  unsigned long long b = (unsigned long long)__double_as_longlong(norm2);
  return (b & ~0xFFFFull) | (unsigned long long)(0xFFFF - col);
}

// Initial column norms: one warp per (problem, eligible column).
__global__ void qr_init_kernel(const QRProb* __restrict__ probs, QRState* __restrict__ st,
                               const int* __restrict__ colprefix, int nprob, int64_t ncols,
                               const double* __restrict__ pool, unsigned char* __restrict__ chosen,
                               double* __restrict__ nu2, double* __restrict__ nuref2) {
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  int p = find_prob(colprefix, nprob, (int)gw);
  const QRProb q = probs[p];
  int col = (int)(gw - colprefix[p]);
  if (lane == 0) chosen[q.col0 + col] = 0;
  if (col >= q.cpiv) return;
  const double* a = pool + q.a + (int64_t)col * q.lda;
  double s = 0.0;
  for (int i = lane; i < q.m; i += 32) s = fma(a[i], a[i], s);
  s = warp_sum(s);
  if (lane == 0) {
    nu2[q.col0 + col] = s;
    nuref2[q.col0 + col] = s;
    atomicMax(&st[p].key[0], pivot_key(s, col));
  }
}

__global__ void qr_reset_kernel(QRState* st, int nprob) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  st[p].done = 0; st[p].k = 0; st[p].r11 = 0.0; st[p].tau = 0.0;
  st[p].key[0] = 0ull; st[p].key[1] = 0ull;
}

// Step j for problem p, by one whole CTA: choose the pivot, build the
// Householder reflector H = I - tau v v^T with H x = beta e_j, store v and tau.
__device__ void qr_pivot_step(int p, const QRProb* __restrict__ probs, QRState* __restrict__ st, int j,
                              double* __restrict__ pool, int* __restrict__ piv,
                              unsigned char* __restrict__ chosen, double* __restrict__ vbuf,
                              int* __restrict__ ndone, DevStatus* dst, int level) {
  __shared__ double red[QR_THREADS / 32];
  __shared__ int s_p, s_stop;
  QRState* S = st + p;
  const int t = threadIdx.x;
  // every early return is preceded by a barrier after the shared flag is
  // read, so the CTA's next problem cannot overwrite it under a slow thread
  if (t == 0) s_stop = S->done;
  __syncthreads();
  const int was_done = s_stop;
  __syncthreads();
  if (was_done) return;
  const QRProb q = probs[p];
  if (t == 0) {
    unsigned long long key = S->key[j & 1];
    int stop = 0;
    if (j >= q.maxk || j >= q.m || j >= q.cpiv || key == 0ull) stop = 1;
    s_p = stop ? -1 : 0xFFFF - (int)(key & 0xFFFFull);
    if (stop) { S->done = 1; S->k = j; atomicAdd(ndone, 1); }
    s_stop = stop;
  }
  __syncthreads();
  const int stop1 = s_stop;
  const int pc = s_p;
  __syncthreads();
  if (stop1) return;
  double* a = pool + q.a + (int64_t)pc * q.lda;
  double s = 0.0;
  for (int i = j + t; i < q.m; i += QR_THREADS) s = fma(a[i], a[i], s);
  s = warp_sum(s);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int w = 0; w < QR_THREADS / 32; w++) tot += red[w];
    double nrm = sqrt(tot);
    if (!(nrm == nrm) || nrm > DBL_MAX) report(dst, RSF_ENUMERIC, level, p, j);
    if (j == 0) S->r11 = nrm;
    int stop = (nrm == 0.0) || (q.tol > 0.0 && nrm <= q.tol * S->r11) || !(nrm == nrm);
    if (stop) {
      S->done = 1; S->k = j; atomicAdd(ndone, 1);
    } else {
      double x0 = a[j];
      double beta = x0 >= 0.0 ? -nrm : nrm;
      double v0 = x0 - beta;
      S->tau = (beta - x0) / beta;
      red[0] = 1.0 / v0;
      a[j] = beta;
      piv[q.col0 + j] = pc;
      chosen[q.col0 + pc] = 1;
      S->key[(j + 1) & 1] = 0ull;
    }
    s_stop = stop;
  }
  __syncthreads();
  if (!s_stop) {
    const double inv_v0 = red[0];
    double* v = vbuf + q.row0;
    if (t == 0) v[j] = 1.0;
    for (int i = j + 1 + t; i < q.m; i += QR_THREADS) {
      v[i] = a[i] * inv_v0;
      a[i] = 0.0;
    }
  }
  __syncthreads();   // red and s_* are reused for the CTA's next problem
}

// Step j for global column gw, by one warp: apply H to the column (if it is
// not chosen) and offer it as the next pivot.  The norm below row j is
// downdated, nu^2 <- nu^2 - a_j^2 (a_j the updated entry in row j, since H is
// orthogonal on rows >= j), and recomputed from the updated column whenever
// the downdate has lost more than half the digits: nu^2 <= sqrt(eps) times
// the norm^2 of the last exact computation (the safeguard of the LAPACK
// pivoted QR, Drmac & Bujanovic 2008).  That saves one of the three fp64
// multiply-adds per element and step.
__device__ __forceinline__ void qr_update_col(int64_t gw, int lane, const QRProb* __restrict__ probs,
                                              QRState* __restrict__ st, const int* __restrict__ colprefix,
                                              const int* __restrict__ colprob, int j, double* __restrict__ pool,
                                              const unsigned char* __restrict__ chosen,
                                              const double* __restrict__ vbuf, double* __restrict__ nu2,
                                              double* __restrict__ nuref2) {
  const int p = colprob[gw];
  if (st[p].done) return;
  const QRProb q = probs[p];
  int col = (int)(gw - colprefix[p]);
  if (chosen[q.col0 + col]) return;
  double* a = pool + q.a + (int64_t)col * q.lda;
  const double* v = vbuf + q.row0;
  double s = 0.0;
  for (int i = j + lane; i < q.m; i += 32) s = fma(v[i], a[i], s);
  s = warp_sum(s) * st[p].tau;
  const bool track = col < q.cpiv;
  double nu = 0.0, nref = 0.0;
  bool recompute = false;
  if (track) {
    const double xj = a[j] - s;   // v[j] = 1
    nref = nuref2[q.col0 + col];
    nu = nu2[q.col0 + col] - xj * xj;
    recompute = !(nu > QR_TOL3Z * nref);
  }
  __syncwarp();   // every lane has read a[j] before lane 0 overwrites it
  double n2 = 0.0;
  for (int i = j + lane; i < q.m; i += 32) {
    double x = fma(-s, v[i], a[i]);
    a[i] = x;
    if (recompute && i > j) n2 = fma(x, x, n2);
  }
  if (recompute) {
    n2 = warp_sum(n2);
    nu = n2;
    nref = n2;
  }
  if (lane == 0 && track) {
    nu2[q.col0 + col] = nu;
    nuref2[q.col0 + col] = nref;
    atomicMax(&st[p].key[(j + 1) & 1], pivot_key(nu, col));
  }
}

// Grid-wide barrier of a cooperative launch (every CTA resident), with a
// bounded wait: after QR_BARRIER_SPINS polls the CTA reports RSF_ETIMEOUT and
// the caller leaves the kernel.  bar[0] counts arrivals, bar[1] is the
// generation.
__device__ bool qr_grid_barrier(unsigned int* bar, unsigned int nblocks, DevStatus* dst, int level) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) + 1u == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (++it > QR_BARRIER_SPINS) {
          ok = 0;
          report(dst, RSF_ETIMEOUT, level, -1, 0);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole column-pivoted QR of a batch in one cooperative launch: per step
// a pivot phase (CTAs over problems) and an update phase (warps over columns),
// separated by grid barriers.  The loop ends after maxsteps steps or once every
// problem is done; ndone changes only in a pivot phase, so every CTA reads the
// same count between the two barriers of a step and all leave together.
__global__ void __launch_bounds__(QR_THREADS) qr_persistent_kernel(
    const QRProb* __restrict__ probs, QRState* __restrict__ st, const int* __restrict__ colprefix,
    const int* __restrict__ colprob, int nprob, int64_t ncols, int maxsteps, double* __restrict__ pool,
    int* __restrict__ piv,
    unsigned char* __restrict__ chosen, double* __restrict__ vbuf, double* __restrict__ nu2,
    double* __restrict__ nuref2, int* __restrict__ ndone, unsigned int* __restrict__ bar, DevStatus* dst,
    int level) {
  const unsigned int nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * QR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)nb * (QR_THREADS / 32);
  for (int j = 0; j <= maxsteps; j++) {
    for (int p = blockIdx.x; p < nprob; p += nb)
      qr_pivot_step(p, probs, st, j, pool, piv, chosen, vbuf, ndone, dst, level);
    if (!qr_grid_barrier(bar, nb, dst, level)) return;
    if (j == maxsteps || *(volatile int*)ndone >= nprob) return;
    for (int64_t gw = wid; gw < ncols; gw += nwarps)
      qr_update_col(gw, lane, probs, st, colprefix, colprob, j, pool, chosen, vbuf, nu2, nuref2);
    if (!qr_grid_barrier(bar, nb, dst, level)) return;
  }
}

// Self-test of the bounded grid barrier: every CTA waits for one more CTA
// than the grid holds, so the wait can only end by its limit.
__global__ void barrier_timeout_probe_kernel(unsigned int* bar, DevStatus* dst) {
  qr_grid_barrier(bar, gridDim.x + 1, dst, -1);
}

int barrier_timeout_selftest(cudaStream_t s) {
  DBuf bar, st;
  bar.alloc(2 * sizeof(unsigned int), s);
  bar.zero();
  st.alloc(sizeof(DevStatus), s);
  st.zero();
  unsigned int* a_bar = bar.as<unsigned int>();
  DevStatus* a_st = st.as<DevStatus>();
  void* args[] = {&a_bar, &a_st};
  RSF_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_timeout_probe_kernel, dim3(2), dim3(QR_THREADS), args, 0,
                                       s));
  ::rsf::g_launches++;
  DevStatus h{};
  d2h(&h, a_st, 1, s);
  sync(s);
  return h.code;
}

void QRBatch::build(const std::vector<QRProb>& p, cudaStream_t s) {
  nprob = (int)p.size();
  std::vector<QRProb> pp = p;
  colprefix_h.assign(nprob + 1, 0);
  ncols = 0; nrows = 0; maxsteps = 0;
  for (int i = 0; i < nprob; i++) {
    RSF_CHECK(pp[i].cpiv <= 0xFFFF, RSF_EINVAL, "qr: too many pivot columns");
    pp[i].col0 = ncols;
    pp[i].row0 = nrows;
    ncols += pp[i].c;
    nrows += pp[i].m;
    colprefix_h[i + 1] = (int)ncols;
    maxsteps = std::max(maxsteps, std::min(pp[i].maxk, std::min(pp[i].m, pp[i].cpiv)));
  }
  RSF_CHECK(ncols < (int64_t)1 << 31, RSF_EINVAL, "qr: too many columns");
  upload(prob, pp, s);
  upload(colprefix, colprefix_h, s);
  {
    // problem of every column (the update phase looks it up once per column)
    std::vector<int> cp(std::max<int64_t>(1, ncols), 0);
    for (int i = 0; i < nprob; i++)
      for (int c = colprefix_h[i]; c < colprefix_h[i + 1]; c++) cp[c] = i;
    upload(colprob, cp, s);
  }
  state.alloc(sizeof(QRState) * std::max(1, nprob), s);
  piv.alloc(sizeof(int) * std::max<int64_t>(1, ncols), s);
  chosen.alloc(std::max<int64_t>(1, ncols), s);
  vbuf.alloc(sizeof(double) * std::max<int64_t>(1, nrows), s);
  nu2.alloc(sizeof(double) * std::max<int64_t>(1, ncols), s);
  nuref2.alloc(sizeof(double) * std::max<int64_t>(1, ncols), s);
  ndone.alloc(sizeof(int) * 4, s);   // [0] problems done, [1..2] the grid barrier
}

// CTAs of the persistent QR kernel that fit on the device at once (cached per
// device; a cooperative launch needs all of them resident).
static int qr_grid_capacity() {
  static int cached[64] = {};
  int dev = 0;
  RSF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int sms = 0, per_sm = 0;
  RSF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RSF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_persistent_kernel, QR_THREADS, 0));
  RSF_CHECK(per_sm > 0, RSF_ECUDA, "qr: the persistent kernel cannot be resident");
  const int cap = sms * per_sm;
  if (dev >= 0 && dev < 64) cached[dev] = cap;
  return cap;
}

void QRBatch::run(double* pool, DevStatus* st, int level, cudaStream_t s) {
  if (nprob == 0) return;
  LAUNCH(qr_reset_kernel, cdiv(nprob, 128), 128, 0, s, state.as<QRState>(), nprob);
  ndone.zero();
  int blocksU = cdiv(ncols * 32, 256);
  LAUNCH(qr_init_kernel, blocksU, 256, 0, s, prob.as<QRProb>(), state.as<QRState>(),
         colprefix.as<int>(), nprob, ncols, pool, chosen.as<unsigned char>(), nu2.as<double>(),
         nuref2.as<double>());
  // one CTA per problem or one warp per column, at most what is resident
  const int64_t want = std::max<int64_t>(nprob, cdiv(ncols, QR_THREADS / 32));
  const int grid = (int)std::min<int64_t>(want, qr_grid_capacity());
  const QRProb* a_probs = prob.as<QRProb>();
  QRState* a_st = state.as<QRState>();
  const int* a_cp = colprefix.as<int>();
  const int* a_cprob = colprob.as<int>();
  int a_nprob = nprob;
  int64_t a_ncols = ncols;
  int a_maxsteps = maxsteps;
  double* a_pool = pool;
  int* a_piv = piv.as<int>();
  unsigned char* a_chosen = chosen.as<unsigned char>();
  double* a_vbuf = vbuf.as<double>();
  double* a_nu2 = nu2.as<double>();
  double* a_nuref2 = nuref2.as<double>();
  int* a_ndone = ndone.as<int>();
  unsigned int* a_bar = reinterpret_cast<unsigned int*>(ndone.as<int>() + 1);
  DevStatus* a_dst = st;
  int a_level = level;
  void* args[] = {&a_probs, &a_st, &a_cp, &a_cprob, &a_nprob, &a_ncols, &a_maxsteps, &a_pool,
                  &a_piv, &a_chosen, &a_vbuf, &a_nu2, &a_nuref2, &a_ndone, &a_bar, &a_dst, &a_level};
  int tu = prof_begin(s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (verbose()) {
    RSF_CUDA(cudaEventCreate(&e0));
    RSF_CUDA(cudaEventCreate(&e1));
    RSF_CUDA(cudaEventRecord(e0, s));
  }
  RSF_CUDA(cudaLaunchCooperativeKernel((const void*)qr_persistent_kernel, dim3(grid), dim3(QR_THREADS), args, 0, s));
  ::rsf::g_launches++;
  prof_end(tu, s, PROF_QR_UPDATE, 0.0, 0.0);
  if (verbose()) {
    RSF_CUDA(cudaEventRecord(e1, s));
    RSF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RSF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    // fp64 flops of the run: per problem and step j < k, the pivot column's
    // norm (m - j) and, per remaining column, a dot and an update (4 (m - j))
    std::vector<QRState> sth(nprob);
    std::vector<QRProb> pph(nprob);
    d2h(sth.data(), state.as<QRState>(), nprob, s);
    d2h(pph.data(), prob.as<QRProb>(), nprob, s);
    sync(s);
    double fl = 0.0;
    for (int i = 0; i < nprob; i++)
      for (int j = 0; j < sth[i].k; j++) fl += 2.0 * (pph[i].m - j) * (1.0 + 2.0 * (pph[i].c - j - 1));
    fprintf(stderr,
            "[rsf] qr batch (level %d): %d problems, %lld columns, %lld rows, %d steps max, %.2f ms, %.3g flop, "
            "%.3f TFLOP/s\n",
            level, nprob, (long long)ncols, (long long)nrows, maxsteps, ms, fl, fl / (ms * 1e9));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
}

// [S, R] split: S in pivot order, R = remaining eligible columns ascending.
__global__ void qr_split_kernel(const QRProb* __restrict__ probs, const QRState* __restrict__ st,
                                const int* __restrict__ piv, const unsigned char* __restrict__ chosen,
                                const int64_t* __restrict__ out0, int* __restrict__ perm,
                                int* __restrict__ kout) {
  const int p = blockIdx.x;
  const QRProb q = probs[p];
  const int k = st[p].k;
  int* o = perm + out0[p];
  if (threadIdx.x == 0) kout[p] = k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) o[i] = piv[q.col0 + i];
  // ordered compaction of the unchosen eligible columns (single warp scan)
  if (threadIdx.x < 32) {
    int lane = threadIdx.x, base = k;
    for (int c0 = 0; c0 < q.cpiv; c0 += 32) {
      int c = c0 + lane;
      int flag = (c < q.cpiv) && !chosen[q.col0 + c];
      unsigned m = __ballot_sync(0xffffffffu, flag);
      if (flag) o[base + __popc(m & ((1u << lane) - 1u))] = c;
      base += __popc(m);
    }
  }
}

void qr_split(const QRBatch& qb, const int64_t* d_out0, int* d_perm, int* d_kout, cudaStream_t s) {
  if (qb.nprob == 0) return;
  LAUNCH(qr_split_kernel, qb.nprob, 128, 0, s, qb.d_prob(), qb.d_state(), qb.d_piv(),
         qb.chosen.as<unsigned char>(), d_out0, d_perm, d_kout);
}

// Back-substitution, one warp per (problem, rhs): column-oriented, in place in
// the output column.  Uses R11[i][jj] = A[i, piv[jj]].
struct TrsmDev {
  int nrhs;
  int64_t rhs0, out0;
};

__global__ void qr_trsm_kernel(const QRProb* __restrict__ probs, const QRState* __restrict__ st,
                               const int* __restrict__ piv, const TrsmDev* __restrict__ tp,
                               const int* __restrict__ prefix, int nprob, int total,
                               const int* __restrict__ rhs, const double* __restrict__ pool,
                               double* __restrict__ outpool, DevStatus* dst, int level) {
  int gw = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (gw >= total) return;
  int p = find_prob(prefix, nprob, gw);
  int s = gw - prefix[p];
  const QRProb q = probs[p];
  const TrsmDev d = tp[p];
  const int k = st[p].k;
  const int* pv = piv + q.col0;
  double* x = outpool + d.out0 + (int64_t)s * k;
  if (d.rhs0 >= 0) {
    int col = rhs[d.rhs0 + s];
    const double* a = pool + q.a + (int64_t)col * q.lda;
    for (int i = lane; i < k; i += 32) x[i] = a[i];
  } else {
    for (int i = lane; i < k; i += 32) x[i] = (i == s) ? 1.0 : 0.0;
  }
  __syncwarp();
  int iend = (d.rhs0 >= 0) ? k - 1 : min(s, k - 1);
  for (int i = k - 1; i > iend; i--) {
    if (lane == 0) x[i] = 0.0;  // identity mode: rows below s are zero
  }
  __syncwarp();
  for (int i = iend; i >= 0; i--) {
    const double* ri = pool + q.a + (int64_t)pv[i] * q.lda;  // column i of R11
    double xi = x[i] / ri[i];
    __syncwarp();
    if (lane == 0) x[i] = xi;
    for (int r = lane; r < i; r += 32) x[r] = fma(-xi, ri[r], x[r]);
    __syncwarp();
  }
}

void qr_trsm(const QRBatch& qb, const std::vector<TrsmProb>& tp, const int* d_rhs,
             double* pool, double* outpool, DevStatus* st, int level, cudaStream_t s) {
  if (qb.nprob == 0) return;
  std::vector<TrsmDev> td(qb.nprob);
  std::vector<int> pre(qb.nprob + 1, 0);
  for (int i = 0; i < qb.nprob; i++) {
    td[i].nrhs = tp[i].nrhs;
    td[i].rhs0 = tp[i].rhs0;
    td[i].out0 = tp[i].out0;
    pre[i + 1] = pre[i] + tp[i].nrhs;
  }
  if (pre[qb.nprob] == 0) return;
  DBuf dtd, dpre;
  upload(dtd, td, s);
  upload(dpre, pre, s);
  LAUNCH(qr_trsm_kernel, cdiv((int64_t)pre[qb.nprob] * 32, 256), 256, 0, s, qb.d_prob(),
         qb.d_state(), qb.d_piv(), dtd.as<TrsmDev>(), dpre.as<int>(), qb.nprob, pre[qb.nprob],
         d_rhs, pool, outpool, st, level);
}

// ============================================================== Cholesky
constexpr int NB = 32;

// Panel p0: factor the diagonal block in shared memory, then solve the
// rows below against it.  One CTA (256 threads) per problem.
__global__ void __launch_bounds__(256) chol_panel_kernel(const CholProb* __restrict__ probs,
                                                         int p0, double* __restrict__ pool,
                                                         DevStatus* dst, int level) {
  const CholProb q = probs[blockIdx.x];
  if (p0 >= q.n) return;
  const int nb = min(NB, q.n - p0);
  double* A = pool + q.a;
  const int ld = q.ld;
  __shared__ double D[NB][NB + 1];
  const int t = threadIdx.x;
  for (int idx = t; idx < nb * nb; idx += 256) {
    int i = idx % nb, j = idx / nb;
    D[i][j] = (i >= j) ? A[(p0 + i) + (int64_t)(p0 + j) * ld] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; j++) {
    if (t == 0) {
      double d = D[j][j];
      if (!(d > 0.0)) {
        report(dst, RSF_ENOTPD, level, q.box, p0 + j);
        d = 1.0;
      }
      D[j][j] = sqrt(d);
    }
    __syncthreads();
    double djj = D[j][j];
    for (int i = j + 1 + t; i < nb; i += 256) D[i][j] /= djj;
    __syncthreads();
    for (int idx = t; idx < nb * nb; idx += 256) {
      int i = idx % nb, c = idx / nb;
      if (c > j && i >= c) D[i][c] = fma(-D[i][j], D[c][j], D[i][c]);
    }
    __syncthreads();
  }
  for (int idx = t; idx < nb * nb; idx += 256) {
    int i = idx % nb, j = idx / nb;
    if (i >= j) A[(p0 + i) + (int64_t)(p0 + j) * ld] = D[i][j];
  }
  // rows below: L21 = A21 D^-T (forward substitution per row)
  for (int i = p0 + nb + t; i < q.n; i += 256) {
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) x[j] = (j < nb) ? A[i + (int64_t)(p0 + j) * ld] : 0.0;
#pragma unroll
    for (int j = 0; j < NB; j++) {
      if (j < nb) {
        double v = x[j];
#pragma unroll
        for (int c = 0; c < NB; c++)
          if (c < j) v = fma(-x[c], D[j][c], v);
        x[j] = v / D[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < NB; j++)
      if (j < nb) A[i + (int64_t)(p0 + j) * ld] = x[j];
  }
}

void cholesky_batched(const std::vector<CholProb>& p, double* pool, DevStatus* st, int level,
                      cudaStream_t s) {
  if (p.empty()) return;
  DBuf dp;
  upload(dp, p, s);
  int nmax = 0;
  for (auto& q : p) nmax = std::max(nmax, q.n);
  for (int p0 = 0; p0 < nmax; p0 += NB) {
    LAUNCH(chol_panel_kernel, (int)p.size(), 256, 0, s, dp.as<CholProb>(), p0, pool, st, level);
    int p1 = p0 + NB;
    if (p1 >= nmax) break;
    std::vector<GemmDesc> gd;
    for (auto& q : p) {
      if (q.n <= p1) continue;
      GemmDesc g{};
      g.M = g.N = q.n - p1;
      g.K = NB;
      g.lda = g.ldb = g.ldc = q.ld;
      g.a = q.a + p1 + (int64_t)p0 * q.ld;       // L21
      g.b = g.a;                                  // L21^T
      g.c = q.a + p1 + (int64_t)p1 * q.ld;
      g.abase = g.bbase = g.cbase = 0;
      g.ta = 0; g.tb = 1; g.triB = 0; g.lowC = 1;
      g.alpha = -1.0; g.beta = 1.0;
      gd.push_back(g);
    }
    if (gd.empty()) continue;
    GemmBatch gb;
    gb.build(gd, s);
    GemmBases b{};
    b.p[0] = pool; b.alpha_scale = 1.0;
    b.sc[0] = b.sc[1] = b.sc[2] = b.sc[3] = 1;
    gb.run(b, s);
  }
}

// ====================================================== triangular inverse
__global__ void lower_inverse_kernel(const TriInvProb* __restrict__ probs, const int* __restrict__ prefix,
                                     int nprob, int total, const double* __restrict__ in,
                                     double* __restrict__ out) {
  int gw = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (gw >= total) return;
  int p = find_prob(prefix, nprob, gw);
  const TriInvProb q = probs[p];
  int j = gw - prefix[p];
  const double* C = in + q.a;
  double* y = out + q.out + (int64_t)j * q.n;
  for (int i = lane; i < q.n; i += 32) y[i] = (i == j) ? 1.0 : 0.0;
  __syncwarp();
  for (int i = j; i < q.n; i++) {
    double yi = y[i] / C[i + (int64_t)i * q.ld];
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int r = i + 1 + lane; r < q.n; r += 32) y[r] = fma(-yi, C[r + (int64_t)i * q.ld], y[r]);
    __syncwarp();
  }
}

void lower_inverse_batched(const std::vector<TriInvProb>& p, const double* in, double* out,
                           cudaStream_t s) {
  if (p.empty()) return;
  std::vector<int> pre(p.size() + 1, 0);
  for (size_t i = 0; i < p.size(); i++) pre[i + 1] = pre[i] + p[i].n;
  if (pre.back() == 0) return;
  DBuf dp, dpre;
  upload(dp, p, s);
  upload(dpre, pre, s);
  LAUNCH(lower_inverse_kernel, cdiv((int64_t)pre.back() * 32, 256), 256, 0, s, dp.as<TriInvProb>(),
         dpre.as<int>(), (int)p.size(), pre.back(), in, out);
}

// ============================================================ small helpers
__global__ void symmetrize_kernel(const SqProb* __restrict__ probs, const int64_t* __restrict__ prefix,
                                  int nprob, int64_t total, double* __restrict__ pool) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const SqProb q = probs[lo];
  int64_t e = g - prefix[lo];
  int i = (int)(e % q.n), j = (int)(e / q.n);
  if (i <= j) return;
  double* A = pool + q.a;
  double a = A[i + (int64_t)j * q.ld], b = A[j + (int64_t)i * q.ld];
  double m = 0.5 * (a + b);
  A[i + (int64_t)j * q.ld] = m;
  A[j + (int64_t)i * q.ld] = m;
}

void symmetrize_batched(const std::vector<SqProb>& p, double* pool, cudaStream_t s) {
  if (p.empty()) return;
  std::vector<int64_t> pre(p.size() + 1, 0);
  for (size_t i = 0; i < p.size(); i++) pre[i + 1] = pre[i] + (int64_t)p[i].n * p[i].n;
  if (pre.back() == 0) return;
  DBuf dp, dpre;
  upload(dp, p, s);
  upload(dpre, pre, s);
  LAUNCH(symmetrize_kernel, cdiv(pre.back(), 256), 256, 0, s, dp.as<SqProb>(), dpre.as<int64_t>(),
         (int)p.size(), pre.back(), pool);
}

__global__ void copy_kernel(const CopyProb* __restrict__ probs, const int64_t* __restrict__ prefix,
                            int nprob, int64_t total, const double* __restrict__ src,
                            double* __restrict__ dst) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const CopyProb q = probs[lo];
  int64_t e = g - prefix[lo];
  int i = (int)(e % q.m), j = (int)(e / q.m);
  double v = q.trans ? src[q.src + j + (int64_t)i * q.lds] : src[q.src + i + (int64_t)j * q.lds];
  dst[q.dst + i + (int64_t)j * q.ldd] = v;
}

void copy_batched(const std::vector<CopyProb>& p, const double* src, double* dst, cudaStream_t s) {
  if (p.empty()) return;
  std::vector<int64_t> pre(p.size() + 1, 0);
  for (size_t i = 0; i < p.size(); i++) pre[i + 1] = pre[i] + (int64_t)p[i].m * p[i].n;
  if (pre.back() == 0) return;
  DBuf dp, dpre;
  upload(dp, p, s);
  upload(dpre, pre, s);
  LAUNCH(copy_kernel, cdiv(pre.back(), 256), 256, 0, s, dp.as<CopyProb>(), dpre.as<int64_t>(),
         (int)p.size(), pre.back(), src, dst);
}

}  // namespace rsf
