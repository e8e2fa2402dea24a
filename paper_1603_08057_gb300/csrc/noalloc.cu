// rsf_solve_noalloc: the multi-right-hand-side solve of rsf_solve with every
// work buffer carved from one file-scope device array instead of allocated.
//
// Who needs it: callers that cannot allocate device memory at solve time --
// code running inside another framework's memory budget (its caching
// allocator has reserved the device memory, so a cudaMalloc would fail or
// fragment that pool), and latency-critical loops that must not pay for an
// allocation's implicit device synchronisation.  The factorization handle
// itself is still built (and allocated) beforehand by rsf_build.
//
// The array lives in every device that loads the library until the process
// exits.  Its device address is looked up once per device, on the first call
// made while that device is current.
#include <mutex>

#include "internal.cuh"

namespace rsf {

// Kernels shared with the allocating paths (solve.cu, api.cu).
__global__ void gather_rows_kernel(const int* __restrict__ src, int64_t nrows, int q,
                                   const double* __restrict__ child, const double* __restrict__ in,
                                   double* __restrict__ out, int cvt);
__global__ void scatter_rows_kernel(const int* __restrict__ src, int64_t nrows, int q,
                                    const double* __restrict__ lev, double* __restrict__ child,
                                    double* __restrict__ out, int cvt);
__global__ void copy_ranges_kernel(const int64_t* __restrict__ rr, int nrr, int q,
                                   const double* __restrict__ from, double* __restrict__ to);
__global__ void to_tree_kernel(const double* __restrict__ B, int64_t ldb, int q, const int* __restrict__ perm,
                               int64_t n, double* __restrict__ X);
__global__ void from_tree_kernel(const double* __restrict__ X, int64_t n, int q, const int* __restrict__ perm,
                                 double* __restrict__ B, int64_t ldb);

static __device__ __align__(256) double g_noalloc_scratch[RSF_NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on device dev, which must be current
// (the symbol lookup resolves on the current device).
double* noalloc_scratch(int dev) {
  RSF_CHECK(dev >= 0 && dev < kMaxDevices, RSF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    RSF_CHECK(e == cudaSuccess && p != nullptr, RSF_ECUDA,
              std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  return g_noalloc_ptr[dev];
}

void level_gemm(const GemmBatch& g, double* X, double* pool, int q, double alpha, int df, cudaStream_t s) {
  GemmBases b{};
  b.p[0] = X; b.p[1] = nullptr; b.p[2] = pool; b.p[3] = nullptr;
  b.sc[0] = q; b.sc[1] = q; b.sc[2] = 1; b.sc[3] = 1;
  b.M = q; b.ld = q; b.alpha_scale = alpha;
  b.df = df == 1 ? 3 : df;   // the tensor-core engine without work buffers
  g.run(b, s);
}
}  // namespace

// Doubles of scratch one call needs: input and output blocks in tree order,
// one block per level and a temporary of the largest level (all nrhs wide).
static int64_t noalloc_need(const rsf_handle_s* h, int nrhs) {
  int64_t rows = 0, maxrows = 0;
  for (const LevelData& Lv : h->levels) {
    rows += Lv.nrows;
    maxrows = std::max(maxrows, Lv.nrows);
  }
  return (int64_t)nrhs * (2 * h->tree_raw->t.n + rows + maxrows);
}

void solve_noalloc(rsf_handle_s* h, double* B, int64_t ldb, int nrhs, int op) {
  cudaStream_t s = h->stream;
  const int64_t n = h->tree_raw->t.n;
  const int q = nrhs;
  const int L = (int)h->levels.size() - 1;
  const int df = h->df;
  const int64_t need = noalloc_need(h, nrhs);
  RSF_CHECK(need <= (int64_t)RSF_NOALLOC_SCRATCH_DOUBLES, RSF_EINVAL,
            "rsf_solve_noalloc: nrhs * (2 n + sum of level rows + largest level) = " + std::to_string(need) +
                " doubles exceeds the scratch of " + std::to_string((int64_t)RSF_NOALLOC_SCRATCH_DOUBLES));
  // The kernels run on the handle's stream, which belongs to the device the
  // handle was built on; the scratch address must be that device's.
  int cur = -1;
  RSF_CUDA(cudaGetDevice(&cur));
  RSF_CHECK(cur == h->device, RSF_EINVAL,
            "rsf_solve_noalloc: the current device (" + std::to_string(cur) + ") is not the handle's device (" +
                std::to_string(h->device) + "); make the handle's device current first");
  double* ws = noalloc_scratch(h->device);
  // carve: Xin | Xout | level blocks | tmp  (nothing needs to start at zero:
  // every element is written before it is read)
  double* Xin = ws;
  double* Xout = Xin + n * q;
  double* Xlev = Xout + n * q;
  std::vector<int64_t> off(L + 2, 0);
  int64_t maxrows = 0;
  for (int l = 0; l <= L; l++) {
    off[l + 1] = off[l] + h->levels[l].nrows;
    maxrows = std::max(maxrows, h->levels[l].nrows);
  }
  double* tmp = Xlev + off[L + 1] * q;
  auto Xl = [&](int l) { return Xlev + off[l] * q; };
  const int cvt = df;
  const int* perm = h->tree_raw->t.perm.as<int>();
  LAUNCH(to_tree_kernel, cdiv(n * q, 256), 256, 0, s, B, ldb, q, perm, n, Xin);

  int up = 0, down = 0, mid = 0;
  switch (op) {
    case RSF_OP_INV: up = 1; down = 1; mid = 0; break;
    case RSF_OP_APPLY: up = 2; down = 2; mid = 1; break;
    case RSF_OP_SQRT: up = 0; down = 2; mid = 2; break;
    case RSF_OP_SQRT_T: up = 2; down = 0; mid = 3; break;
    case RSF_OP_INV_SQRT: up = 1; down = 0; mid = 4; break;
    case RSF_OP_INV_SQRT_T: up = 0; down = 1; mid = 5; break;
    default: fail(RSF_EINVAL, "unknown op");
  }
  for (int l = L; l >= 0; l--) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrows == 0) continue;
    const double* child = (l < L) ? Xl(l + 1) : nullptr;
    LAUNCH(gather_rows_kernel, cdiv(Lv.nrows, 8), 256, 0, s, Lv.src.as<int>(), Lv.nrows, q, child, Xin, Xl(l), cvt);
    if (l == 0) break;
    double* F = Lv.fpool.as<double>();
    if (up == 1) {
      level_gemm(Lv.gRS_T, Xl(l), F, q, -1.0, df, s);
      level_gemm(Lv.gSR_Et, Xl(l), F, q, -1.0, df, s);
    } else if (up == 2) {
      level_gemm(Lv.gSR_Tt, Xl(l), F, q, 1.0, df, s);
      level_gemm(Lv.gRS_E, Xl(l), F, q, 1.0, df, s);
    }
  }
  for (int l = 0; l <= L; l++) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrr == 0) continue;
    double* F = Lv.fpool.as<double>();
    double* x = Xl(l);
    auto prod = [&](int v, bool from_tmp) {
      GemmBases b{};
      b.p[0] = from_tmp ? tmp : x; b.p[1] = from_tmp ? x : tmp; b.p[2] = F; b.p[3] = nullptr;
      b.sc[0] = q; b.sc[1] = q; b.sc[2] = 1; b.sc[3] = 1;
      b.M = q; b.ld = q; b.alpha_scale = 1.0;
      b.df = df == 1 ? 3 : df;
      Lv.gMid[v].run(b, s);
    };
    auto copy_to_tmp = [&]() {
      LAUNCH(copy_ranges_kernel, Lv.nrr, 256, 0, s, Lv.rr.as<int64_t>(), Lv.nrr, q, x, tmp);
    };
    switch (mid) {
      case 0: prod(0, false); prod(1, true); break;
      case 1:
        if (h->spd) { prod(2, false); prod(3, true); }
        else { copy_to_tmp(); prod(4, true); }
        break;
      case 2: copy_to_tmp(); prod(3, true); break;
      case 3: copy_to_tmp(); prod(2, true); break;
      case 4: copy_to_tmp(); prod(0, true); break;
      case 5: copy_to_tmp(); prod(1, true); break;
    }
  }
  for (int l = 0; l <= L; l++) {
    LevelData& Lv = h->levels[l];
    if (Lv.nrows == 0) continue;
    double* F = Lv.fpool.as<double>();
    if (l > 0) {
      if (down == 1) {
        level_gemm(Lv.gRS_E, Xl(l), F, q, -1.0, df, s);
        level_gemm(Lv.gSR_Tt, Xl(l), F, q, -1.0, df, s);
      } else if (down == 2) {
        level_gemm(Lv.gSR_Et, Xl(l), F, q, 1.0, df, s);
        level_gemm(Lv.gRS_T, Xl(l), F, q, 1.0, df, s);
      }
    }
    double* child = (l < L) ? Xl(l + 1) : nullptr;
    LAUNCH(scatter_rows_kernel, cdiv(Lv.nrows, 8), 256, 0, s, Lv.src.as<int>(), Lv.nrows, q, Xl(l), child, Xout,
           cvt);
  }
  LAUNCH(from_tree_kernel, cdiv(n * q, 256), 256, 0, s, Xout, n, q, perm, B, ldb);
}

}  // namespace rsf
