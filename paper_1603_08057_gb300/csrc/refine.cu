// Iterative refinement of alpha = Sigma^-1 z (Algorithm 1, first line;
// Eq. (loglikelihood)): the RSF solve gives alpha to the factorization's
// accuracy (eps_fact); one sweep alpha <- alpha + F^-1 (z - Sigma alpha) with
// the residual computed against the exact kernel matrix brings z^T alpha to
// the accuracy of that residual.  The residual needs Sigma alpha, an O(n^2)
// matvec evaluated on the fly (Sigma is never stored), in arithmetic finer
// than the factorization's error:
//
//   * Matern nu = 1/2, 3/2, 5/2: df64 (fp32-pair, ~48-bit) arithmetic on the
//     fp32 pipes, which issue 64x more operations per clock than the fp64
//     pipe on this GPU.  exp(-a) is computed from the mathematics: argument
//     reduction a = k ln2 + rho with ln 2 split into three parts (Cody and
//     Waite's method), then exp(-rho) = (exp(-rho / 16))^16 with a degree-7
//     Taylor polynomial for |rho / 16| <= 0.022 (truncation below 2e-18) and
//     four squarings ("scaling and squaring", J.-M. Muller, Elementary
//     Functions, ch. 11); the square root is one Newton step in df64 from the
//     fp32 root;
//   * rational quadratic with an integer shape alpha = 1..8: df64 as well,
//     (1 + r^2 / (2 alpha l^2))^-alpha from a df64 reciprocal (one Newton
//     step from the fp32 one) raised by repeated multiplication;
//   * every other kernel (Matern nu = 1, rational quadratic with other
//     alpha): fp64 with the library's fp64 kernel evaluation (O(n^2) fp64
//     work: slow at large n, so not run by default, see refine_sweeps).
// Both accumulate each row's sum in df64 (error-free products and sums), so
// the residual carries ~1e-14 relative rounding of sum_j |K_ij alpha_j|.
//
// Rows and columns are in tree order; in a forest (independent point sets)
// a row only sums over its own set, which is contiguous in tree order.
#include <cmath>

#include "df64.cuh"
#include "internal.cuh"

namespace rsf {

namespace {
constexpr int RT = 256;   // rows per CTA (one per thread) and columns per shared-memory tile

// ---------------------------------------------------------------- df64 math
__device__ __forceinline__ df64 d_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 d_neg(df64 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 d_sub(df64 a, df64 b) { return df_add(a, d_neg(b)); }
// sqrt of a >= 0: fp32 root, then one Newton correction in df64
__device__ __forceinline__ df64 d_sqrt(df64 a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float y = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(y, y);
  const float pe = __fmaf_rn(y, y, -p);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);   // a - y^2 (a.hi - p exact)
  return df_fast_two_sum(y, __fdiv_rn(d, __fmul_rn(2.f, y)));
}

// ln 2 = L0 + L1 + L2: L0 carries 12 significant bits (k L0 exact for
// k < 2^11), L1 the next 24, L2 the rest; values from ln 2 =
// 0.693147180559945309417232121458176568...
struct Ln2Parts {
  float L0, L1, L2;
};
__constant__ Ln2Parts c_ln2;
// 1/m! for m = 0..7 as df64 pairs
__constant__ df64 c_invfact[8];

// exp(-a) for a >= 0 (0 beyond a = 86, where it is below 2^-124)
__device__ __forceinline__ df64 d_exp_neg(df64 a) {
  if (a.hi > 86.f) return {0.f, 0.f};
  const float k = rintf(__fmul_rn(a.hi, 1.4426950408889634f));
  // rho = a - k ln2: a.hi - k L0 is exact (both on a grid of 2^-17 at most,
  // |difference| < 1); k L1 exactly as a df64 product; k L2 is tiny
  const float r0 = __fsub_rn(a.hi, __fmul_rn(k, c_ln2.L0));
  const float p1 = __fmul_rn(k, c_ln2.L1);
  const float e1 = __fmaf_rn(k, c_ln2.L1, -p1);
  df64 rho = df_add({r0, a.lo}, {-p1, -e1});
  rho = df_add(rho, {-__fmul_rn(k, c_ln2.L2), 0.f});
  // exp(-rho) = exp(-rho/16)^16
  const df64 s = {-rho.hi * 0.0625f, -rho.lo * 0.0625f};
  df64 p = c_invfact[7];
#pragma unroll
  for (int m = 6; m >= 0; m--) p = df_add(d_mul(p, s), c_invfact[m]);
#pragma unroll
  for (int i = 0; i < 4; i++) p = d_mul(p, p);
  // times 2^-k (exact; k <= 125)
  const float sc = __uint_as_float((uint32_t)(127 - (int)k) << 23);
  return {p.hi * sc, p.lo * sc};
}

// Off-diagonal Matern correlation times s2, in df64: nu = 1/2: e^-a,
// a = r/l; 3/2: (1 + a) e^-a, a = sqrt3 r/l; 5/2: (1 + a + a^2/3) e^-a,
// a = sqrt5 r/l (Sec. 1 Eq. (matern) at half-integer nu).
struct MaternDF {
  int family;
  int aniso;    // scale dx by ax and dy by ay (Sec. 5.1; unit length scale in c)
  df64 ax, ay;
  df64 c;       // a = c r (Matern); 1 / (2 alpha l^2) (rational quadratic)
  df64 s2;
  df64 third;   // 1/3
  int alpha;    // rational quadratic: integer shape
};

__device__ __forceinline__ df64 d_recip(df64 u) {
  const float y = __fdiv_rn(1.f, u.hi);
  // t = 1 - u y, evaluated with the exact product u.hi y
  const float p = __fmul_rn(u.hi, y);
  const float pe = __fmaf_rn(u.hi, y, -p);
  const float t = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(u.lo, y));
  return df_fast_two_sum(y, __fmul_rn(y, t));
}

// s2 (1 + r^2 c)^-alpha for the rational quadratic with integer alpha
__device__ __forceinline__ df64 rq_df(const MaternDF& m, df64 r2) {
  const df64 u = df_add({1.f, 0.f}, d_mul(r2, m.c));
  const df64 inv = d_recip(u);
  df64 p = inv;
  for (int i = 1; i < m.alpha; i++) p = d_mul(p, inv);
  return d_mul(m.s2, p);
}

__device__ __forceinline__ df64 matern_df(const MaternDF& m, df64 r) {
  const df64 a = d_mul(m.c, r);
  const df64 e = d_exp_neg(a);
  df64 poly = {1.f, 0.f};
  if (m.family == RSF_MATERN32) {
    poly = df_add(poly, a);
  } else if (m.family == RSF_MATERN52) {
    poly = df_add(df_add(poly, a), d_mul(d_mul(a, a), m.third));
  }
  return d_mul(m.s2, d_mul(poly, e));
}

// Row set range [j0, j1) of tree position i in a forest of nsets sets.
__device__ __forceinline__ void set_range(const int64_t* __restrict__ set_off, int nsets, int64_t i, int64_t& j0,
                                          int64_t& j1) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (set_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  j0 = set_off[lo];
  j1 = set_off[lo + 1];
}

// r = z - Sigma x, one row per thread; DF selects the df64 Matern path.
template <bool DF>
__global__ void __launch_bounds__(RT) residual_kernel(const double* __restrict__ xt, const double* __restrict__ z,
                                                      const double* __restrict__ x, const int64_t* __restrict__ set_off,
                                                      int nsets, int64_t n, KernelParams kp, MaternDF md,
                                                      double* __restrict__ r) {
  __shared__ double sx[RT], sy[RT], sv[RT];
  __shared__ df64 dx_s[RT], dy_s[RT], dv_s[RT];   // the same tile as df64 pairs (DF path)
  __shared__ unsigned long long s_lo, s_hi;
  const int t = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * RT + t;
  int64_t j0 = 0, j1 = 0;
  double xi = 0.0, yi = 0.0;
  if (t == 0) {
    s_lo = ~0ull;
    s_hi = 0ull;
  }
  __syncthreads();
  if (i < n) {
    set_range(set_off, nsets, i, j0, j1);
    xi = xt[2 * i];
    yi = xt[2 * i + 1];
    atomicMin(&s_lo, (unsigned long long)j0);
    atomicMax(&s_hi, (unsigned long long)j1);
  }
  __syncthreads();
  const int64_t c0 = (int64_t)s_lo, c1 = (int64_t)s_hi;
  const df64 xid = df_from_double(xi), yid = df_from_double(yi);
  dfacc acc = {0.f, 0.f};
  double acc64 = 0.0, comp = 0.0;   // fp64 path: Kahan-compensated sum
  for (int64_t jt = c0; jt < c1; jt += RT) {
    const int64_t j = jt + t;
    if (j < c1) {
      if (DF) {
        dx_s[t] = df_from_double(xt[2 * j]);
        dy_s[t] = df_from_double(xt[2 * j + 1]);
        dv_s[t] = df_from_double(x[j]);
      } else {
        sx[t] = xt[2 * j];
        sy[t] = xt[2 * j + 1];
        sv[t] = x[j];
      }
    }
    __syncthreads();
    const int jn = c1 - jt < RT ? (int)(c1 - jt) : RT;
    if (i < n) {
      for (int jj = 0; jj < jn; jj++) {
        const int64_t jg = jt + jj;
        if (jg < j0 || jg >= j1) continue;
        if (DF) {
          df64 v;
          if (jg == i) {
            v = df_from_double(kernel_diag(kp));
          } else {
            df64 dx = d_sub(xid, dx_s[jj]);
            df64 dy = d_sub(yid, dy_s[jj]);
            if (md.aniso) {
              dx = d_mul(dx, md.ax);
              dy = d_mul(dy, md.ay);
            }
            const df64 r2 = df_add(d_mul(dx, dx), d_mul(dy, dy));
            v = md.family == RSF_RQ ? rq_df(md, r2) : matern_df(md, d_sqrt(r2));
          }
          df_mac(acc, v, dv_s[jj]);
        } else {
          const double k = jg == i ? kernel_diag(kp) : kernel_pair(kp, xi, yi, sx[jj], sy[jj]);
          const double y = fma(k, sv[jj], -comp);
          const double tsum = acc64 + y;
          comp = (tsum - acc64) - y;
          acc64 = tsum;
        }
      }
    }
    __syncthreads();
  }
  if (i < n) r[i] = z[i] - (DF ? df_to_double(df_of_acc(acc)) : acc64);
}

// y_i = sum_j K(xs_i, x_j) v_j for m new points xs against n points x (both
// row-major, 2 doubles per point): the cross-covariance matvec of the
// conditional mean (no nugget: different observations), fp64 with a
// Kahan-compensated sum.
__global__ void __launch_bounds__(RT) cross_matvec_kernel(const double* __restrict__ xt, const double* __restrict__ v,
                                                          int64_t n, const double* __restrict__ xs, int64_t m,
                                                          KernelParams kp, double* __restrict__ y) {
  __shared__ double sx[RT], sy[RT], sv[RT];
  const int t = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * RT + t;
  const double xi = i < m ? xs[2 * i] : 0.0, yi = i < m ? xs[2 * i + 1] : 0.0;
  double acc = 0.0, comp = 0.0;
  for (int64_t jt = 0; jt < n; jt += RT) {
    const int64_t j = jt + t;
    if (j < n) {
      sx[t] = xt[2 * j];
      sy[t] = xt[2 * j + 1];
      sv[t] = v[j];
    }
    __syncthreads();
    const int jn = n - jt < RT ? (int)(n - jt) : RT;
    if (i < m)
      for (int jj = 0; jj < jn; jj++) {
        const double k = kernel_pair(kp, xi, yi, sx[jj], sy[jj]);
        const double yk = fma(k, sv[jj], -comp);
        const double tsum = acc + yk;
        comp = (tsum - acc) - yk;
        acc = tsum;
      }
    __syncthreads();
  }
  if (i < m) y[i] = acc;
}

__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y[g] += x[g];
}

bool g_df_consts[64] = {};

// The constant-memory tables of the df64 exp, once per device.
void init_df_consts() {
  int dev = 0;
  RSF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && g_df_consts[dev]) return;
  // ln 2 to 36 significant digits, split into fp32 parts
  const long double ln2 = 0.693147180559945309417232121458176568L;
  Ln2Parts p;
  p.L0 = std::ldexp(std::nearbyint(std::ldexp((double)ln2, 12)), -12);   // 12 bits: 2^-12 grid
  const long double rem1 = ln2 - (long double)p.L0;
  p.L1 = (float)rem1;
  p.L2 = (float)(rem1 - (long double)p.L1);
  df64 inv[8];
  long double f = 1.0L;
  for (int m = 0; m < 8; m++) {
    if (m > 0) f *= m;
    const long double v = 1.0L / f;
    inv[m].hi = (float)v;
    inv[m].lo = (float)(v - (long double)inv[m].hi);
  }
  RSF_CUDA(cudaMemcpyToSymbol(c_ln2, &p, sizeof p));
  RSF_CUDA(cudaMemcpyToSymbol(c_invfact, inv, sizeof inv));
  if (dev >= 0 && dev < 64) g_df_consts[dev] = true;
}

df64 host_df(double v) {
  df64 d;
  d.hi = (float)v;
  d.lo = (float)(v - (double)d.hi);
  return d;
}
}  // namespace

bool residual_uses_df64(const KernelParams& kp) {
  if (kp.family == RSF_RQ) return kp.alpha >= 1.0 && kp.alpha <= 8.0 && kp.alpha == std::floor(kp.alpha);
  return kp.family == RSF_MATERN12 || kp.family == RSF_MATERN32 || kp.family == RSF_MATERN52;
}

void kernel_residual(rsf_handle_s* F, const double* zt, const double* xt_vec, double* rt, int force_fp64) {
  const TreeData& T = F->tree_raw->t;
  cudaStream_t s = F->stream;
  const int64_t n = T.n;
  KernelParams kp = F->kp;
  kp.which = 0;
  MaternDF md{};
  md.family = kp.family;
  const double c = kp.family == RSF_MATERN32 ? std::sqrt(3.0) : kp.family == RSF_MATERN52 ? std::sqrt(5.0) : 1.0;
  const double l = kp.aniso ? 1.0 : kp.l;   // anisotropic: unit length on the scaled differences
  md.aniso = kp.aniso;
  md.ax = host_df(kp.aniso ? 1.0 / kp.l : 1.0);
  md.ay = host_df(kp.aniso ? 1.0 / kp.l2 : 1.0);
  md.c = host_df(kp.family == RSF_RQ ? 1.0 / (2.0 * kp.alpha * l * l) : c / l);
  md.alpha = kp.family == RSF_RQ ? (int)kp.alpha : 0;
  md.s2 = host_df(kp.s2);
  md.third = host_df(1.0 / 3.0);
  const bool df = residual_uses_df64(kp) && !force_fp64;
  if (df) init_df_consts();
  if (df)
    LAUNCH(residual_kernel<true>, cdiv(n, RT), RT, 0, s, T.xt.as<double>(), zt, xt_vec, T.set_off_d.as<int64_t>(),
           T.nsets, n, kp, md, rt);
  else
    LAUNCH(residual_kernel<false>, cdiv(n, RT), RT, 0, s, T.xt.as<double>(), zt, xt_vec, T.set_off_d.as<int64_t>(),
           T.nsets, n, kp, md, rt);
}

void cross_matvec(KernelParams kp, const double* x, const double* v, int64_t n, const double* xs, int64_t m,
                  double* y, cudaStream_t s) {
  kp.which = 0;
  if (m > 0) LAUNCH(cross_matvec_kernel, cdiv(m, RT), RT, 0, s, x, v, n, xs, m, kp, y);
}

void add_into(double* y, const double* x, int64_t n, cudaStream_t s) {
  if (n > 0) LAUNCH(axpy_kernel, cdiv(n, 256), 256, 0, s, y, x, n);
}

}  // namespace rsf
