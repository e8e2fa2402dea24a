// Shared infrastructure of the RSF library: error handling, stream-ordered
// device buffers, the device status word and launch accounting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsf.h"

namespace rsf {

// ---------------------------------------------------------------- errors
struct Error {
  rsf_status code;
  std::string msg;
};

void set_error(const std::string& msg);
[[noreturn]] void fail(rsf_status code, const std::string& msg);

#define RSF_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      ::rsf::fail(e_ == cudaErrorMemoryAllocation ? RSF_ENOMEM : RSF_ECUDA,  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

#define RSF_CHECK(cond, code, msg)                  \
  do {                                              \
    if (!(cond)) ::rsf::fail((code), (msg));        \
  } while (0)

// Launch accounting: every kernel launch of the library goes through LAUNCH,
// which counts it and checks the launch error.
extern int64_t g_launches;
#define LAUNCH(kernel, grid, block, smem, stream, ...)                       \
  do {                                                                        \
    dim3 g_ = (grid);                                                         \
    if (g_.x > 0 && g_.y > 0 && g_.z > 0) {                                   \
      kernel<<<g_, (block), (smem), (stream)>>>(__VA_ARGS__);                 \
      ::rsf::g_launches++;                                                    \
      RSF_CUDA(cudaGetLastError());                                           \
    }                                                                         \
  } while (0)

// Optional per-category kernel timing: CUDA events recorded on the launching
// stream around instrumented launches, with the launch's algorithmic flops.
enum ProfCat {
  PROF_GEMM = 0, PROF_QR_UPDATE = 1 /* the whole persistent pivoted QR */, PROF_QR_PIVOT = 2 /* unused */,
  // phases (spans of many launches)
  PROF_PEEL_APPLY = 3, PROF_PEEL_SUB = 4, PROF_PEEL_QR = 5, PROF_PEEL_REST = 6, PROF_FACTOR = 7,
  PROF_GEMM_DF = 8,  // the GEMM kernel in df64 arithmetic (PROF_GEMM: fp64)
  PROF_GEMM_TC = 9,  // the tensor-core GEMM on df64 operands (tcgemm.cu)
  PROF_NCAT = 10
};
// Diagnostics to stderr when the environment variable RSF_VERBOSE is set.
bool verbose();
bool prof_enabled();
// Returns a token for prof_end (or -1 when profiling is off).
int prof_begin(cudaStream_t s);
void prof_end(int token, cudaStream_t s, int cat, double flops, double bytes);

// Device status word written by kernels on numerical failure:
// [0] code (rsf_status), [1] level, [2] box, [3] detail.
struct DevStatus {
  int code, level, box, detail;
};

__device__ __forceinline__ void report(DevStatus* st, int code, int level, int box, int detail) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->level = level;
    st->box = box;
    st->detail = detail;
  }
}

// ---------------------------------------------------------- device memory
// Allocator hook set through rsf_set_allocator (null members: the default,
// stream-ordered cudaMallocAsync / cudaFreeAsync).
struct AllocHook {
  rsf_alloc_fn alloc = nullptr;
  rsf_free_fn free = nullptr;
  void* ctx = nullptr;
};
AllocHook alloc_hook();

// Stream-ordered allocation; the owner frees on the same stream, through the
// allocator that provided the memory.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  rsf_free_fn hfree = nullptr;   // non-null: memory from the hook
  void* hctx = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s; hfree = o.hfree; hctx = o.hctx;
      o.p = nullptr; o.bytes = 0; o.hfree = nullptr; o.hctx = nullptr;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t nbytes, cudaStream_t stream) {
    release();
    s = stream;
    bytes = nbytes;
    if (nbytes == 0) return;
    const AllocHook h = alloc_hook();
    if (h.alloc) {
      p = h.alloc(nbytes, (void*)stream, h.ctx);
      if (!p) {
        bytes = 0;
        RSF_CHECK(false, RSF_ENOMEM, "the allocator hook returned NULL for " + std::to_string(nbytes) + " bytes");
      }
      hfree = h.free;
      hctx = h.ctx;
    } else {
      RSF_CUDA(cudaMallocAsync(&p, nbytes, stream));
    }
  }
  void zero() {
    if (bytes) RSF_CUDA(cudaMemsetAsync(p, 0, bytes, s));
  }
  void release() {
    if (p) {
      if (hfree) hfree(p, bytes, (void*)s, hctx);
      else cudaFreeAsync(p, s);
    }
    p = nullptr;
    bytes = 0;
    hfree = nullptr;
    hctx = nullptr;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

template <class T>
inline void h2d(T* dst, const T* src, size_t count, cudaStream_t s) {
  if (count) RSF_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
}
template <class T>
inline void d2h(T* dst, const T* src, size_t count, cudaStream_t s) {
  if (count) RSF_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
}
// Upload a host vector into a fresh device buffer.
template <class T>
inline void upload(DBuf& b, const std::vector<T>& v, cudaStream_t s) {
  b.alloc(v.size() * sizeof(T), s);
  h2d(b.as<T>(), v.data(), v.size(), s);
}
inline void sync(cudaStream_t s) { RSF_CUDA(cudaStreamSynchronize(s)); }

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace rsf
