// Batched ragged GEMM on the fifth-generation tensor cores (tcgen05) with
// fp64-class accuracy, for the mixed-precision solves and peeling products
// (Sec. 2.3.2 applies and solves, Sec. 3 peeling products).
//
// Operands and result are df64 pairs (df64.cuh), exactly as for the CUDA-core
// df64 GEMM; the descriptors are the same GemmDesc batches.  The product is
// formed from exact bf16 "slices" (the splitting scheme of Ozaki, Ogita,
// Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer.
// Algorithms 59 (2012), here with bf16 slices and fp32 accumulation):
//
//   * per K-block of at most KB = 64 terms, every row m of op(A) gets the
//     power of two 2^E_m > max_k |A_mk| and every column n of op(B) the power
//     2^F_n > max_k |B_kn|;
//   * a = A_mk / 2^E_m in (-1, 1) is cut into S = 7 slices a_j, each a
//     multiple of 2^-7(j+1) with at most 8 significant bits (exact in bf16):
//     a_j = round-to-nearest of the remainder onto the grid 2^-7(j+1); the
//     remainder after S slices is below 2^-50;
//   * slice products a_s b_t are exact in fp32 and multiples of
//     2^-7(s+t+2); all products of one "diagonal" d = s + t share that grid,
//     so one fp32 TMEM accumulator per diagonal sums them EXACTLY as long as
//     the integer sum stays below 2^24: |a_0|, |b_0| <= 128 units, later
//     slices <= 65, so a diagonal gains at most 16640 + 4225 (d - 1) <=
//     37765 units per term and 64 terms stay far below 2^24 (up to 444 would);
//   * diagonals d >= S are dropped (the truncation error is ~S 2^-7(S+1) of
//     2^(E_m+F_n) per term, below the df64 rounding of the inputs);
//   * the epilogue reads the S diagonals from TMEM, sums them by TwoSum into
//     a df64 value,
//     scales by 2^(E_m + F_n) and adds alpha times it to C (the first block
//     also applies beta), in df64 like the CUDA-core df64 kernel.
//
// Work split (one persistent CTA per SM over the 128 x 64 output tiles of the
// batch; 9 warps):
//   * warps 0-7 load a whole K-block (64 terms: 32 A values of one row and 16
//     B values of one column per thread, every load issued at once, so the
//     block's exponents come from registers without a second pass over
//     memory), slice it into one of three shared-memory stages per 16-term
//     chunk (canonical K-major, no-swizzle core-matrix layout), copy the C
//     values the block updates into shared memory asynchronously
//     (cp.async) while the MMAs finish, and run the block's epilogue (each
//     thread one TMEM lane and 32 columns);
//   * warp 8 allocates the 512 TMEM columns (the S = 7 accumulators of 64
//     columns); its lane 0 issues the 28 tcgen05.mma instructions of a chunk
//     (M = 128, N = 64, K = 16, bf16 x bf16 -> fp32) and commits to the
//     mbarriers that free the stage and that hand a finished block to the
//     epilogue.
// Measured on GB300 (rsf_selftest_gemm, 4096 x 4096 x 384 and 2048^3):
// 6-6.5 TFLOP/s fp64-equivalent including the operand copies, 1.5x the
// CUDA-core df64 kernel at the same accuracy class.  The producer warps
// bound it (per 64-term block: one ~8k-cycle load round trip, ~8k cycles of
// slicing, ~13k of epilogue); the tensor pipe is mostly idle.
// Every wait is bounded (a few seconds): on expiry the CTA records
// RSF_ETIMEOUT, drains its own MMAs, frees its TMEM and returns.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "dense.cuh"
#include "df64.cuh"

namespace rsf {

namespace tc {
constexpr int BM = 128, BN = TC_BN, KC = 16, KB = 64, S = 7, NST = 3;
constexpr int PW = 8;                          // slicing / epilogue warps
constexpr int NPROD = PW * 32;
constexpr int NTHREADS = NPROD + 32;           // + the MMA warp
constexpr int A_SLICE = BM * KC * 2;           // bytes of one bf16 slice of an A stage
constexpr int B_SLICE = BN * KC * 2;
constexpr int STAGE = S * (A_SLICE + B_SLICE);
constexpr int A_LBO = (BM / 8) * 128;          // bytes between k-groups of 8 (core matrices)
constexpr int B_LBO = (BN / 8) * 128;
constexpr int TMEM_COLS = 512;
constexpr int CBUF = BM * BN * 8;             // the C tile (df64) staged for the epilogue
constexpr int AUX = 4096;
constexpr int SMEM = NST * STAGE + CBUF + AUX + 1024; // + alignment slack
constexpr unsigned long long WAIT_NS = 4000000000ull;
static_assert(S * BN <= TMEM_COLS, "the S accumulators must fit the allocated TMEM columns");
static_assert(KB == 4 * KC && BM * KB == NPROD * 32 && BN * KB == NPROD * 16, "thread ownership of a K-block");
static_assert(SMEM <= 232448, "shared memory of one CTA");
}  // namespace tc

__device__ DevStatus g_tc_status;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on expiry or when
// another thread of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  uint64_t t0 = 0;
  for (uint32_t it = 1;; it++) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      const uint64_t now = gtimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > tc::WAIT_NS) return false;
    }
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride byte offset
// (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Power of two strictly above every |v| with max |hi| = m (0 for m = 0),
// clamped to [-126, 126] so that 2^E and 2^-E are normal fp32 numbers
// (operands of magnitude >= 2^126 are outside this engine's range).
__device__ __forceinline__ int block_exponent(float m) {
  if (!(m > 0.f)) return 0;
  const int e = (int)((__float_as_uint(m) >> 23) & 0xFF) - 126;
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// Next slice of the remainder h + l (|h + l| < 2^-7j) on the grid
// 2^-7(j+1): g = round(h + l) to the grid (adding and subtracting
// 1.5 x 2^(23 - 7(j+1)) rounds to that grid in one fp32 addition), then the
// remainder h - g, which is exact (both are multiples of the finer of their
// grids and the difference is at most half a grid step).
__device__ __forceinline__ float next_slice(float& h, float l, float magic) {
  const float t = __fadd_rn(h, l);
  const float y = __fadd_rn(t, magic);
  const float g = __fsub_rn(y, magic);
  h = __fsub_rn(h, g);
  return g;
}
// Two slices (fp32 values with at most 8 significant bits) packed as bf16x2
// by truncation, which is exact for them: low half the first.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  return __byte_perm(__float_as_uint(lo_elem), __float_as_uint(hi_elem), 0x7632);
}

__device__ __forceinline__ float slice_magic(int j) {
  // 1.5 x 2^(23 - 7 (j + 1))
  return 1.5f * pow2f(16 - 7 * j);
}

// The S slices of 8 consecutive k of one row: slice j as 8 bf16 (16 bytes,
// one core-matrix row) at dst + j * slice_bytes.
__device__ __forceinline__ void slice_store(float (&hh)[8], const float (&ll)[8], uint8_t* dst, int slice_bytes) {
#pragma unroll
  for (int j = 0; j < tc::S; j++) {
    const float mg = slice_magic(j);
    float s8[8];
#pragma unroll
    for (int i = 0; i < 8; i++) s8[i] = next_slice(hh[i], ll[i], mg);
    uint4 w;
    w.x = pack_bf16x2(s8[0], s8[1]);
    w.y = pack_bf16x2(s8[2], s8[3]);
    w.z = pack_bf16x2(s8[4], s8[5]);
    w.w = pack_bf16x2(s8[6], s8[7]);
    *reinterpret_cast<uint4*>(dst + j * slice_bytes) = w;
  }
}

// Base array i of the launch (a select chain keeps the parameter struct in
// registers instead of indexing it through local memory).
__device__ __forceinline__ double* base_ptr(const GemmBases& b, int i) {
  return i == 0 ? b.p[0] : i == 1 ? b.p[1] : i == 2 ? b.p[2] : b.p[3];
}
__device__ __forceinline__ int64_t base_scale(const GemmBases& b, int i) {
  return i == 0 ? b.sc[0] : i == 1 ? b.sc[1] : i == 2 ? b.sc[2] : b.sc[3];
}

__global__ void __launch_bounds__(tc::NTHREADS, 1)
    tc_gemm_kernel(const GemmDesc* __restrict__ descs, const int2* __restrict__ ntile, int ntilesN, int mtiles,
                   GemmBases bases) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float2* sC = reinterpret_cast<float2*>(sm + NST * STAGE);   // [BN][BM]: C(row, col) at col * BM + row
  uint8_t* aux = sm + NST * STAGE + CBUF;
  int* sExpB = reinterpret_cast<int*>(aux);                 // [2][BN] (by K-block parity)
  float* sPartA = reinterpret_cast<float*>(sExpB + 2 * BN); // [NPROD]
  float* sPartB = sPartA + NPROD;                           // [NPROD]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sPartB + NPROD);
  // bars: full[NST], empty[NST], accf, acce, drain, prod
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2 * NST + 4);
  volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);
  const uint32_t bFull = su32(bars), bEmpty = su32(bars + NST), bAccF = su32(bars + 2 * NST),
                 bAccE = su32(bars + 2 * NST + 1), bDrain = su32(bars + 2 * NST + 2),
                 bProd = su32(bars + 2 * NST + 3);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp < PW;
  if (tid == 0) {
    for (int i = 0; i < NST; i++) {
      mbar_init(bFull + 8 * i, NPROD);
      mbar_init(bEmpty + 8 * i, 1);
    }
    mbar_init(bAccF, 1);
    mbar_init(bAccE, NPROD);
    mbar_init(bDrain, 1);
    mbar_init(bProd, NPROD);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == PW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(sTmem)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(BM >> 4) << 24);
  // Ownership of a K-block (64 terms = 8 k-groups of 8):
  //   A: row r, k-groups kh, kh + 2, kh + 4, kh + 6 (kh = 0, 1);
  //   B: column cb, k-groups qb, qb + 4 (qb = 0..3);
  // chunk c of the block takes k-groups 2c and 2c + 1, so every thread
  // slices one A group of each chunk (slot kh) and the B threads with
  // qb + 4j in {2c, 2c + 1} one B group.  In the epilogue the
  // thread reads TMEM lane r (its warp's lane quarter) and columns
  // 32 kh .. 32 kh + 31.
  const int r = tid & (BM - 1), kh = (tid >> 7) & 1;
  const int cb = tid & (BN - 1), qb = (tid >> 6) & 3;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  uint32_t chunk_ctr = 0, blk_ctr = 0;
  bool issued = false;   // the MMA thread issued MMAs (drained on abort)
  const int ntiles = ntilesN * mtiles;
  for (int tile = blockIdx.x; tile < ntiles && !*sAbort; tile += gridDim.x) {
    const int tn = tile / mtiles, tm = tile - tn * mtiles;
    const int2 pn = ntile[tn];
    const GemmDesc d = descs[pn.x];
    const int M = d.M >= 0 ? d.M : bases.M;
    const int N = d.N, K = d.K;
    const int n0 = pn.y;
    const int m0 = tm * BM;
    if (m0 >= M || n0 >= N) continue;
    if (d.lowC && n0 > m0 + BM - 1) continue;
    const int lda = d.lda >= 0 ? d.lda : bases.ld;
    const int ldb = d.ldb >= 0 ? d.ldb : bases.ld;
    const int ldc = d.ldc >= 0 ? d.ldc : bases.ld;
    const double* __restrict__ A = base_ptr(bases, d.abase) + d.a * base_scale(bases, d.abase) + d.m0;
    const double* __restrict__ Bm = base_ptr(bases, d.bbase) + d.b * base_scale(bases, d.bbase);
    double* __restrict__ C = base_ptr(bases, d.cbase) + d.c * base_scale(bases, d.cbase) + d.m0;
    int k0 = 0, k1 = K;
    if (d.triB == 1) k0 = min(n0, K);
    if (d.triB == 2) k1 = min(K, n0 + BN);
    const int nblk = k1 > k0 ? (k1 - k0 + KB - 1) / KB : 0;
    const int nvalid = min(BN, N - n0);
    const bool masktri = d.triB != 0 && !d.gatherK && !d.gatherN;
    const double alpha = d.alpha * bases.alpha_scale, beta = d.beta;
    const int gm = m0 + r;
    const bool rowok = gm < M;
    const int gnb = n0 + cb;

    auto addrA = [&](int gk) -> const double* {
      if (d.gatherK) return A + gm + (int64_t)bases.kidx[d.kofs + gk] * lda;
      return d.ta ? A + gk + (int64_t)gm * lda : A + gm + (int64_t)gk * lda;
    };
    auto addrB = [&](int gk) -> const double* {
      if (d.gatherK) return Bm + (bases.kidx[d.kofs + gk] - d.kb0) + (int64_t)gnb * ldb;
      if (d.gatherN) return Bm + (bases.kidx[d.nofs + gnb] - d.nb0) + (int64_t)gk * ldb;
      return d.tb ? Bm + gnb + (int64_t)gk * ldb : Bm + gk + (int64_t)gnb * ldb;
    };
    auto zeroB = [&](int gk) -> bool {
      return masktri && ((d.triB == 1 && gk < gnb) || (d.triB == 2 && gk > gnb));
    };

    for (int b = 0; b < nblk && !*sAbort; b++, blk_ctr++) {
      const int kb0 = k0 + b * KB, kb1 = min(k1, kb0 + KB), nk = kb1 - kb0;
      const int nch = (nk + KC - 1) / KC;
      const int eb = blk_ctr & 1;
      if (producer) {
        // ---- every load of the block at once (its exponents need all of it)
        float2 a[32], bv[16];
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const int k = kb0 + (kh + 2 * j) * 8 + i;
            a[j * 8 + i] = (rowok && k < kb1) ? *reinterpret_cast<const float2*>(addrA(k)) : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const int k = kb0 + (qb + 4 * j) * 8 + i;
            bv[j * 8 + i] = (gnb < N && k < kb1 && !zeroB(k)) ? *reinterpret_cast<const float2*>(addrB(k))
                                                               : make_float2(0.f, 0.f);
          }
        float ma = 0.f, mb = 0.f;
#pragma unroll
        for (int i = 0; i < 32; i++) ma = fmaxf(ma, fabsf(a[i].x));
#pragma unroll
        for (int i = 0; i < 16; i++) mb = fmaxf(mb, fabsf(bv[i].x));
        sPartA[tid] = ma;
        sPartB[tid] = mb;
        // every producer's partial maxima (a bounded wait: a barrier that
        // another producer's abort could leave forever short is not used)
        mbar_arrive(bProd);
        if (!mbar_wait(bProd, blk_ctr & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        const int eA = block_exponent(fmaxf(sPartA[r], sPartA[r + BM]));
        const int eB = block_exponent(fmaxf(fmaxf(sPartB[cb], sPartB[cb + BN]),
                                            fmaxf(sPartB[cb + 2 * BN], sPartB[cb + 3 * BN])));
        if (tid < BN) sExpB[eb * BN + tid] = eB;
        const float scA = pow2f(-eA), scB = pow2f(-eB);
        // ---- slice the (up to four) chunks of the block into the stages
#pragma unroll
        for (int c = 0; c < 4; c++) {
          if (c >= nch) break;
          const uint32_t cc = chunk_ctr + c;
          const int stage = cc % NST;
          const uint32_t use = cc / NST;
          if (use > 0 && !mbar_wait(bEmpty + 8 * stage, (use - 1) & 1, sAbort)) {
            *sAbort = 1;
            break;
          }
          uint8_t* sA = sm + stage * STAGE;
          uint8_t* sB = sA + S * A_SLICE;
          {  // A group kh + 2c -> chunk slot kh
            float hh[8], ll[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
              hh[i] = a[c * 8 + i].x * scA;
              ll[i] = a[c * 8 + i].y * scA;
            }
            slice_store(hh, ll, sA + kh * A_LBO + (r >> 3) * 128 + (r & 7) * 16, A_SLICE);
          }
          // B group qb + 4j -> chunk slot qb + 4j - 2c, for the threads whose
          // group lies in this chunk
#pragma unroll
          for (int j = 0; j < 2; j++) {
            const int slot = qb + 4 * j - 2 * c;
            if (slot == 0 || slot == 1) {
              float hh[8], ll[8];
#pragma unroll
              for (int i = 0; i < 8; i++) {
                hh[i] = bv[j * 8 + i].x * scB;
                ll[i] = bv[j * 8 + i].y * scB;
              }
              slice_store(hh, ll, sB + slot * B_LBO + (cb >> 3) * 128 + (cb & 7) * 16, B_SLICE);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(bFull + 8 * stage);
        }
        if (*sAbort) break;
        // ---- epilogue: load the C values this block updates while the last
        // MMAs run; the first block writes alpha v + beta C, later blocks add
        // alpha v
        const bool first = b == 0;
        const bool rd = !first || beta != 0.0;
        // the C values go to shared memory by asynchronous copies (no
        // registers held while the MMAs finish)
        if (rd) {
#pragma unroll 4
          for (int j = 0; j < 32; j++) {
            const int col = kh * 32 + j, gn = n0 + col;
            const bool ok = rowok && gn < N && !(d.lowC && gm < gn);
            const int64_t cnn = ok ? (d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn) : 0;
            const double* src = ok ? C + gm + cnn * ldc : C;
            const uint32_t dst = su32(sC + col * BM + r);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0)
                         : "memory");
          }
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        if (!mbar_wait(bAccF, blk_ctr & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        tc_fence_after();
        if (rd) asm volatile("cp.async.wait_all;\n" ::: "memory");
        const float scr = pow2f(eA);
#pragma unroll
        for (int q8 = 0; q8 < 4; q8++) {
          const int col = kh * 32 + q8 * 8;
          if (col < nvalid) {
            float D[S][8];
#pragma unroll
            for (int dd = 0; dd < S; dd++) tmem_ld8(tl + dd * BN + col, D[dd]);
            tmem_ld_wait();
#pragma unroll
            for (int j2 = 0; j2 < 8; j2++) {
              const int gn = n0 + col + j2;
              if (!rowok || gn >= N || (d.lowC && gm < gn)) continue;
              // exact-ish sum of the diagonals, smallest first (TwoSum into
              // hi, the errors into lo)
              float hi = D[S - 1][j2], lo = 0.f;
#pragma unroll
              for (int dd = S - 2; dd >= 0; dd--) {
                const float x = D[dd][j2];
                const float sm2 = __fadd_rn(hi, x);
                const float v = __fsub_rn(sm2, hi);
                lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(sm2, v)), __fsub_rn(x, v)));
                hi = sm2;
              }
              const float scn = pow2f(sExpB[eb * BN + col + j2]);
              df64 t = df_fast_two_sum(hi, lo);
              t.hi = (t.hi * scr) * scn;
              t.lo = (t.lo * scr) * scn;
              t = df_scale(t, (float)alpha);
              const float2 oc = sC[(col + j2) * BM + r];
              df64 o = {oc.x, oc.y};
              if (first && beta != 1.0) o = df_scale(o, (float)beta);
              if (rd) t = df_add(t, o);
              const int64_t cnn = d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn;
              *reinterpret_cast<float2*>(C + gm + cnn * ldc) = make_float2(t.hi, t.lo);
            }
          }
        }
        tc_fence_before();
        mbar_arrive(bAccE);
      } else if (warp == PW && lane == 0) {
        // ---- MMA issue: all slice products with s + t < S, K = 16 each
        if (blk_ctr > 0 && !mbar_wait(bAccE, (blk_ctr - 1) & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        tc_fence_after();
        uint32_t inited = 0;
        for (int c = 0; c < nch; c++) {
          const uint32_t cc = chunk_ctr + c;
          const int stage = cc % NST;
          if (!mbar_wait(bFull + 8 * stage, (cc / NST) & 1, sAbort)) {
            *sAbort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t aBase = su32(sm + stage * STAGE), bBase = aBase + S * A_SLICE;
          const int ksteps = (min(KC, nk - c * KC) + 15) / 16;
          for (int kk = 0; kk < ksteps; kk++) {
#pragma unroll
            for (int s1 = 0; s1 < S; s1++) {
              const uint64_t ad = smem_desc(aBase + s1 * A_SLICE + kk * 2 * A_LBO, A_LBO, 128);
#pragma unroll
              for (int t1 = 0; t1 < S - s1; t1++) {
                const int dd = s1 + t1;
                const uint64_t bd = smem_desc(bBase + t1 * B_SLICE + kk * 2 * B_LBO, B_LBO, 128);
                mma_bf16(tmem + dd * BN, ad, bd, idesc, (inited >> dd) & 1u);
                inited |= 1u << dd;
              }
            }
          }
          issued = true;
          mma_commit(bEmpty + 8 * stage);
        }
        if (*sAbort) break;
        mma_commit(bAccF);
      }
      chunk_ctr += nch;
    }
    if (*sAbort) break;
    if (producer && nblk == 0 && beta != 1.0 && rowok) {
      // no K terms (empty or masked range): C = beta C
      for (int j2 = 0; j2 < 32; j2++) {
        const int gn = n0 + kh * 32 + j2;
        if (gn >= N || (d.lowC && gm < gn)) continue;
        const int64_t cnn = d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn;
        float2* pc2 = reinterpret_cast<float2*>(C + gm + cnn * ldc);
        df64 o = {0.f, 0.f};
        if (beta != 0.0) {
          const float2 v = *pc2;
          o = df_scale({v.x, v.y}, (float)beta);
        }
        *pc2 = make_float2(o.hi, o.lo);
      }
    }
  }

  // ---- teardown: on abort record the timeout and drain this CTA's MMAs
  if (*sAbort && tid == 0) report(&g_tc_status, RSF_ETIMEOUT, -1, blockIdx.x, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == PW) {
    if (lane == 0 && *sAbort && issued) {
      mma_commit(bDrain);
      volatile int never = 0;
      mbar_wait(bDrain, 0, &never);
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
  }
}

// ================================================= pre-sliced engine
// The same products with the slicing taken out of the GEMM: a slicing kernel
// cuts every operand element once into its S bf16 slices, already in the
// shared-memory stage layout (one A block = the S slices of 128 rows x 16
// terms, 28,672 bytes; one B block = 64 columns x 16 terms, 14,336 bytes),
// with one exponent per row of op(A) (column of op(B)) and superblock of
// TC_SBK = 384 terms.  The GEMM kernel then copies whole blocks into its
// stages with bulk asynchronous copies (one loader thread, completion on the
// stage's mbarrier) and sums a whole superblock of 24 chunks in the tensor
// memory before one epilogue: the integer sums of a diagonal stay exact
// (384 terms of at most 37,765 units stay below 2^24), so the exponents'
// coarser range only moves where the last slice's grid falls (2^-49 of the
// row's and column's largest value over the superblock instead of over 64
// terms).  Every element is sliced once instead of once per output tile
// that reads it, and the epilogue runs once per 384 terms instead of per 64.
namespace tc6 {
constexpr int CPS = TC_SBK / tc::KC;              // chunks per superblock
constexpr int A_BLK = tc::S * tc::A_SLICE;        // bytes of one A chunk block
constexpr int B_BLK = tc::S * tc::B_SLICE;
constexpr int NTHREADS = tc::NPROD + 64;          // + the MMA warp + the loader warp
constexpr int SLICE_THREADS = 128;
static_assert(TC_SBK % tc::KC == 0 && TC_SBK % 64 == 0 && TC_SBK <= 444, "superblock of exact sums");
static_assert(TC_BM == tc::BM && TC_KC == tc::KC, "tile shape");
}  // namespace tc6

// op(A)[gm, gk] of a descriptor (gm, gk in range) as a df64 pair
__device__ __forceinline__ float2 tc_load_a(const GemmDesc& d, const GemmBases& b, const double* A, int lda, int gm,
                                            int gk) {
  const double* p = d.gatherK ? A + gm + (int64_t)b.kidx[d.kofs + gk] * lda
                              : (d.ta ? A + gk + (int64_t)gm * lda : A + gm + (int64_t)gk * lda);
  return *reinterpret_cast<const float2*>(p);
}
// op(B)[gk, gn] (in range and not masked)
__device__ __forceinline__ float2 tc_load_b(const GemmDesc& d, const GemmBases& b, const double* Bm, int ldb, int gk,
                                            int gn) {
  const double* p = d.gatherK  ? Bm + (b.kidx[d.kofs + gk] - d.kb0) + (int64_t)gn * ldb
                    : d.gatherN ? Bm + (b.kidx[d.nofs + gn] - d.nb0) + (int64_t)gk * ldb
                    : d.tb      ? Bm + gn + (int64_t)gk * ldb
                                : Bm + gk + (int64_t)gn * ldb;
  return *reinterpret_cast<const float2*>(p);
}

// One work item per block: (descriptor, 128-row tile, superblock) of op(A)
// with one thread per row, or ((descriptor, 64-column tile) entry,
// superblock) of op(B) with one thread per column.  Pass 1 finds the
// exponent, pass 2 writes the slices chunk by chunk (zeros past K, past the
// rows or columns, and in the masked triangle of op(B)).
__global__ void __launch_bounds__(tc6::SLICE_THREADS) tc_slice_kernel(
    const GemmDesc* __restrict__ descs, const TcDescPlan* __restrict__ dplan, int nprob, const int2* __restrict__ ntile,
    const TcEntryPlan* __restrict__ eplan, int nent, int mtL, int64_t itemsA, int64_t items, GemmBases bases,
    uint8_t* __restrict__ abuf, int* __restrict__ ea, uint8_t* __restrict__ bbuf, int* __restrict__ eb) {
  using namespace tc;
  const int t = threadIdx.x;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    if (item < itemsA) {
      int lo = 0, hi = nprob - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dplan[mid].pi + dplan[mid].qi * mtL <= item) lo = mid;
        else hi = mid - 1;
      }
      const TcDescPlan q = dplan[lo];
      const GemmDesc d = descs[lo];
      const int64_t local = item - (q.pi + q.qi * mtL);
      const int mt = (int)(local / q.nsb), sb = (int)(local % q.nsb);
      const int M = d.M >= 0 ? d.M : bases.M, K = d.K;
      const int lda = d.lda >= 0 ? d.lda : bases.ld;
      const double* A = base_ptr(bases, d.abase) + d.a * base_scale(bases, d.abase) + d.m0;
      const int gm = mt * BM + t;
      const bool ok = gm < M;
      const int k0 = sb * TC_SBK, k1 = min(K, k0 + TC_SBK);
      float mx = 0.f;
      if (ok) {
        int k = k0;
        for (; k + 8 <= k1; k += 8) {
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; i++) v[i] = fabsf(tc_load_a(d, bases, A, lda, gm, k + i).x);
#pragma unroll
          for (int i = 0; i < 8; i++) mx = fmaxf(mx, v[i]);
        }
        for (; k < k1; k++) mx = fmaxf(mx, fabsf(tc_load_a(d, bases, A, lda, gm, k).x));
      }
      const int e = block_exponent(mx);
      ea[q.pe + q.qe * mtL + (int64_t)gm * q.nsb + sb] = e;
      const float sc = pow2f(-e);
      for (int ch = k0 / KC; ch * KC < k1; ch++) {
        uint8_t* blk = abuf + (q.pa + q.qa * mtL + (int64_t)mt * q.nch + ch) * (int64_t)tc6::A_BLK;
#pragma unroll
        for (int g = 0; g < 2; g++) {
          float hh[8], ll[8];
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const int k = ch * KC + g * 8 + i;
            const float2 v = (ok && k < k1) ? tc_load_a(d, bases, A, lda, gm, k) : make_float2(0.f, 0.f);
            hh[i] = v.x * sc;
            ll[i] = v.y * sc;
          }
          slice_store(hh, ll, blk + g * A_LBO + (t >> 3) * 128 + (t & 7) * 16, A_SLICE);
        }
      }
    } else {
      // op(B): column c = t mod 64; the two thread halves take the first and
      // second half of the superblock's chunks and share the exponent
      __shared__ float s_mx[tc6::SLICE_THREADS];
      const int64_t bi = item - itemsA;
      int lo = 0, hi = nent - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (eplan[mid].pib <= bi) lo = mid;
        else hi = mid - 1;
      }
      const TcEntryPlan p = eplan[lo];
      const int2 en = ntile[lo];
      const GemmDesc d = descs[en.x];
      const TcDescPlan q = dplan[en.x];
      const int sb = (int)(bi - p.pib);
      const int N = d.N, K = d.K;
      const int ldb = d.ldb >= 0 ? d.ldb : bases.ld;
      const double* Bm = base_ptr(bases, d.bbase) + d.b * base_scale(bases, d.bbase);
      const int c = t & (TC_BN - 1), half = t / TC_BN;
      const int gn = en.y + c;
      const bool ok = gn < N;
      const bool masktri = d.triB != 0 && !d.gatherK && !d.gatherN;
      const int k0 = sb * TC_SBK, k1 = min(K, k0 + TC_SBK);
      const int nchs = (k1 - k0 + KC - 1) / KC, hch = (nchs + 1) / 2;
      const int c0 = k0 / KC + (half ? hch : 0), c1 = k0 / KC + (half ? nchs : hch);
      auto val = [&](int k) -> float2 {
        if (!ok || k >= k1 || (masktri && ((d.triB == 1 && k < gn) || (d.triB == 2 && k > gn))))
          return make_float2(0.f, 0.f);
        return tc_load_b(d, bases, Bm, ldb, k, gn);
      };
      float mx = 0.f;
      for (int ch = c0; ch < c1; ch++) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = fabsf(val(ch * KC + i).x);
#pragma unroll
        for (int i = 0; i < 16; i++) mx = fmaxf(mx, v[i]);
      }
      s_mx[t] = mx;
      __syncthreads();
      const int e = block_exponent(fmaxf(s_mx[c], s_mx[c + TC_BN]));
      __syncthreads();   // s_mx is rewritten by the block's next item
      if (half == 0) eb[p.be + (int64_t)c * q.nsb + sb] = e;
      const float sc = pow2f(-e);
      for (int ch = c0; ch < c1; ch++) {
        uint8_t* blk = bbuf + (p.bblk + ch) * (int64_t)tc6::B_BLK;
#pragma unroll
        for (int g = 0; g < 2; g++) {
          float hh[8], ll[8];
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const float2 v = val(ch * KC + g * 8 + i);
            hh[i] = v.x * sc;
            ll[i] = v.y * sc;
          }
          slice_store(hh, ll, blk + g * B_LBO + (c >> 3) * 128 + (c & 7) * 16, B_SLICE);
        }
      }
    }
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// The GEMM on pre-sliced operands.  Warps 0-7 run the epilogues (one per
// superblock of the tile: TMEM lane r, 32 columns each, as in the engine
// above), warp 8 lane 0 issues the MMAs, warp 9 lane 0 the bulk copies of
// the A and B blocks of every chunk into the three stages.
__global__ void __launch_bounds__(tc6::NTHREADS, 1)
    tc_gemm_pre_kernel(const GemmDesc* __restrict__ descs, const TcDescPlan* __restrict__ dplan,
                       const int2* __restrict__ ntile, const TcEntryPlan* __restrict__ eplan, int ntilesN,
                       int mtiles, int mtL, GemmBases bases, const uint8_t* __restrict__ abuf,
                       const int* __restrict__ ea, const uint8_t* __restrict__ bbuf, const int* __restrict__ eb) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float2* sC = reinterpret_cast<float2*>(sm + NST * STAGE);   // [BN][BM]: C(row, col) at col * BM + row
  uint8_t* aux = sm + NST * STAGE + CBUF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(aux);
  // bars: full[NST], empty[NST], accf, acce, drain, prod
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 2 * NST + 4);
  volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);
  int* sExpB = reinterpret_cast<int*>(aux + 256);            // [2][BN] by unit parity
  const uint32_t bFull = su32(bars), bEmpty = su32(bars + NST), bAccF = su32(bars + 2 * NST),
                 bAccE = su32(bars + 2 * NST + 1), bDrain = su32(bars + 2 * NST + 2),
                 bProd = su32(bars + 2 * NST + 3);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp < PW;
  const bool mma_thread = warp == PW && lane == 0;
  const bool load_thread = warp == PW + 1 && lane == 0;
  if (tid == 0) {
    for (int i = 0; i < NST; i++) {
      mbar_init(bFull + 8 * i, 1);
      mbar_init(bEmpty + 8 * i, 1);
    }
    mbar_init(bAccF, 1);
    mbar_init(bAccE, NPROD);
    mbar_init(bDrain, 1);
    mbar_init(bProd, NPROD);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == PW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(sTmem)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(BM >> 4) << 24);
  const int r = tid & (BM - 1), kh = (tid >> 7) & 1;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  uint32_t chunk_ctr = 0, blk_ctr = 0;
  bool issued = false;          // the MMA thread issued MMAs (drained on abort)
  int last_use[NST];            // the loader's last use of every stage (-1: none)
#pragma unroll
  for (int i = 0; i < NST; i++) last_use[i] = -1;
  const int ntiles = ntilesN * mtiles;
  for (int tile = blockIdx.x; tile < ntiles && !*sAbort; tile += gridDim.x) {
    const int tn = tile / mtiles, tm = tile - tn * mtiles;
    const int2 pn = ntile[tn];
    const GemmDesc d = descs[pn.x];
    const int M = d.M >= 0 ? d.M : bases.M;
    const int N = d.N, K = d.K;
    const int n0 = pn.y;
    const int m0 = tm * BM;
    if (m0 >= M || n0 >= N) continue;
    if (d.lowC && n0 > m0 + BM - 1) continue;
    const TcDescPlan q = dplan[pn.x];
    const TcEntryPlan pe = eplan[tn];
    const int ldc = d.ldc >= 0 ? d.ldc : bases.ld;
    double* __restrict__ C = base_ptr(bases, d.cbase) + d.c * base_scale(bases, d.cbase) + d.m0;
    int k0 = 0, k1 = K;
    if (d.triB == 1) k0 = min(n0, K);
    if (d.triB == 2) k1 = min(K, n0 + BN);
    const int ch0 = k0 / KC, ch1 = k1 > k0 ? (k1 + KC - 1) / KC : ch0;
    const int sb0 = ch0 / tc6::CPS, nunits = ch1 > ch0 ? (ch1 - 1) / tc6::CPS - sb0 + 1 : 0;
    const int nvalid = min(BN, N - n0);
    const double alpha = d.alpha * bases.alpha_scale, beta = d.beta;
    const int gm = m0 + r;
    const bool rowok = gm < M;
    const int64_t ablk0 = q.pa + q.qa * mtL + (int64_t)tm * q.nch;

    for (int u = 0; u < nunits && !*sAbort; u++, blk_ctr++) {
      const int sb = sb0 + u;
      const int cA = max(ch0, sb * tc6::CPS), cB = min(ch1, (sb + 1) * tc6::CPS), nch = cB - cA;
      if (load_thread) {
        // ---- bulk copies of the unit's chunks into the stages
        for (int c = 0; c < nch; c++) {
          const uint32_t cc = chunk_ctr + c;
          const int stage = cc % NST;
          const uint32_t use = cc / NST;
          if (use > 0 && !mbar_wait(bEmpty + 8 * stage, (use - 1) & 1, sAbort)) {
            *sAbort = 1;
            break;
          }
          const uint32_t full = bFull + 8 * stage;
          const uint32_t dA = su32(sm + stage * STAGE);
          mbar_expect_tx(full, (uint32_t)(tc6::A_BLK + tc6::B_BLK));
          bulk_g2s(dA, abuf + (ablk0 + cA + c) * (int64_t)tc6::A_BLK, tc6::A_BLK, full);
          bulk_g2s(dA + tc6::A_BLK, bbuf + (pe.bblk + cA + c) * (int64_t)tc6::B_BLK, tc6::B_BLK, full);
          last_use[stage] = (int)use;
        }
      } else if (mma_thread) {
        // ---- MMAs of the unit: all slice products with s + t < S, summed
        // over its chunks in the S diagonal accumulators
        if (blk_ctr > 0 && !mbar_wait(bAccE, (blk_ctr - 1) & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        tc_fence_after();
        uint32_t inited = 0;
        for (int c = 0; c < nch; c++) {
          const uint32_t cc = chunk_ctr + c;
          const int stage = cc % NST;
          if (!mbar_wait(bFull + 8 * stage, (cc / NST) & 1, sAbort)) {
            *sAbort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t aBase = su32(sm + stage * STAGE), bBase = aBase + S * A_SLICE;
#pragma unroll
          for (int s1 = 0; s1 < S; s1++) {
            const uint64_t ad = smem_desc(aBase + s1 * A_SLICE, A_LBO, 128);
#pragma unroll
            for (int t1 = 0; t1 < S - s1; t1++) {
              const int dd = s1 + t1;
              const uint64_t bd = smem_desc(bBase + t1 * B_SLICE, B_LBO, 128);
              mma_bf16(tmem + dd * BN, ad, bd, idesc, (inited >> dd) & 1u);
              inited |= 1u << dd;
            }
          }
          issued = true;
          mma_commit(bEmpty + 8 * stage);
        }
        if (*sAbort) break;
        mma_commit(bAccF);
      } else if (producer) {
        // ---- epilogue of the unit: C values by asynchronous copies while
        // the MMAs run; the first unit writes alpha v + beta C, later units
        // add alpha v
        const bool first = u == 0;
        const bool rd = !first || beta != 0.0;
        // the unit's column exponents, staged once (double-buffered by unit
        // parity; a producer writes unit u + 2's copy only after every
        // producer has arrived for unit u + 1, i.e. finished unit u)
        const int eb2 = (int)(blk_ctr & 1);
        if (tid < BN) sExpB[eb2 * BN + tid] = eb[pe.be + (int64_t)tid * q.nsb + sb];
        mbar_arrive(bProd);
        if (!mbar_wait(bProd, blk_ctr & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        if (rd) {
#pragma unroll 4
          for (int j = 0; j < 32; j++) {
            const int col = kh * 32 + j, gn = n0 + col;
            const bool ok = rowok && gn < N && !(d.lowC && gm < gn);
            const int64_t cnn = ok ? (d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn) : 0;
            const double* src = ok ? C + gm + cnn * ldc : C;
            const uint32_t dst = su32(sC + col * BM + r);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0)
                         : "memory");
          }
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        const int eA = ea[q.pe + q.qe * mtL + (int64_t)gm * q.nsb + sb];
        if (!mbar_wait(bAccF, blk_ctr & 1, sAbort)) {
          *sAbort = 1;
          break;
        }
        tc_fence_after();
        if (rd) asm volatile("cp.async.wait_all;\n" ::: "memory");
        const float scr = pow2f(eA);
#pragma unroll
        for (int q8 = 0; q8 < 4; q8++) {
          const int col = kh * 32 + q8 * 8;
          if (col < nvalid) {
            float D[S][8];
#pragma unroll
            for (int dd = 0; dd < S; dd++) tmem_ld8(tl + dd * BN + col, D[dd]);
            tmem_ld_wait();
#pragma unroll
            for (int j2 = 0; j2 < 8; j2++) {
              const int gn = n0 + col + j2;
              if (!rowok || gn >= N || (d.lowC && gm < gn)) continue;
              float hi = D[S - 1][j2], lo = 0.f;
#pragma unroll
              for (int dd = S - 2; dd >= 0; dd--) {
                const float x = D[dd][j2];
                const float sm2 = __fadd_rn(hi, x);
                const float v = __fsub_rn(sm2, hi);
                lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(sm2, v)), __fsub_rn(x, v)));
                hi = sm2;
              }
              const float scn = pow2f(sExpB[eb2 * BN + col + j2]);
              df64 t = df_fast_two_sum(hi, lo);
              t.hi = (t.hi * scr) * scn;
              t.lo = (t.lo * scr) * scn;
              t = df_scale(t, (float)alpha);
              const float2 oc = sC[(col + j2) * BM + r];
              df64 o = {oc.x, oc.y};
              if (first && beta != 1.0) o = df_scale(o, (float)beta);
              if (rd) t = df_add(t, o);
              const int64_t cnn = d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn;
              *reinterpret_cast<float2*>(C + gm + cnn * ldc) = make_float2(t.hi, t.lo);
            }
          }
        }
        tc_fence_before();
        mbar_arrive(bAccE);
      }
      chunk_ctr += nch;
    }
    if (*sAbort) break;
    if (producer && nunits == 0 && beta != 1.0 && rowok) {
      // no K terms (empty or masked range): C = beta C
      for (int j2 = 0; j2 < 32; j2++) {
        const int gn = n0 + kh * 32 + j2;
        if (gn >= N || (d.lowC && gm < gn)) continue;
        const int64_t cnn = d.gatherN ? (int64_t)bases.kidx[d.nofs + gn] : (int64_t)gn;
        float2* pc2 = reinterpret_cast<float2*>(C + gm + cnn * ldc);
        df64 o = {0.f, 0.f};
        if (beta != 0.0) {
          const float2 v = *pc2;
          o = df_scale({v.x, v.y}, (float)beta);
        }
        *pc2 = make_float2(o.hi, o.lo);
      }
    }
  }

  // ---- teardown: on abort record the timeout, let this CTA's bulk copies
  // land and drain its MMAs before the tensor memory is freed
  if (*sAbort && tid == 0) report(&g_tc_status, RSF_ETIMEOUT, -1, blockIdx.x, 0);
  if (load_thread) {
    volatile int never = 0;
    for (int i = 0; i < NST; i++)
      if (last_use[i] >= 0) mbar_wait(bFull + 8 * i, (uint32_t)last_use[i] & 1u, &never);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == PW) {
    if (lane == 0 && *sAbort && issued) {
      mma_commit(bDrain);
      volatile int never = 0;
      mbar_wait(bDrain, 0, &never);
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
  }
}

// ------------------------------------------------------------------ host
static int tc_sm_count() {
  static int cnt[64] = {0};
  int dev = 0;
  RSF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cnt[dev]) {
    RSF_CUDA(cudaDeviceGetAttribute(&cnt[dev], cudaDevAttrMultiProcessorCount, dev));
    RSF_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM));
    RSF_CUDA(cudaFuncSetAttribute(tc_gemm_pre_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM));
  }
  return cnt[dev];
}

void tc_gemm_run(const GemmBatch& g, const GemmBases& b, int M, cudaStream_t s) {
  const int mtiles = cdiv(M, tc::BM);
  const int64_t ntiles = (int64_t)g.ntilesN_tc * mtiles;
  if (ntiles == 0) return;
  RSF_CHECK(ntiles < (1ll << 31), RSF_EINVAL, "tensor-core gemm: too many tiles");
  // persistent: one CTA per SM (its shared memory and all 512 TMEM columns)
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)tc_sm_count());
  LAUNCH(tc_gemm_kernel, grid, tc::NTHREADS, tc::SMEM, s, g.desc.as<GemmDesc>(), g.ntile_tc.as<int2>(), g.ntilesN_tc,
         mtiles, b);
}

void tc_gemm_pre_run(const GemmBatch& g, const GemmBases& b, int M, cudaStream_t s) {
  const int mtiles = cdiv(M, tc::BM);
  const int64_t ntiles = (int64_t)g.ntilesN_tc * mtiles;
  if (ntiles == 0) return;
  RSF_CHECK(ntiles < (1ll << 31), RSF_EINVAL, "tensor-core gemm: too many tiles");
  const int sms = tc_sm_count();
  if (!g.tc_dplan.p && !g.tc_dplan_h.empty()) {
    upload(g.tc_dplan, g.tc_dplan_h, s);
    upload(g.tc_eplan, g.tc_eplan_h, s);
  }
  const int mtL = g.anyLaunchM ? cdiv(std::max(b.M, 0), tc::BM) : 0;
  const int64_t itemsA = g.tc_pi + g.tc_qi * mtL, items = itemsA + g.tc_pib;
  const int64_t ablk = g.tc_pa + g.tc_qa * mtL, nea = g.tc_pe + g.tc_qe * mtL;
  // the slices and exponents of this launch (stream-ordered work buffers);
  // when every K is 0 there is nothing to slice, but the GEMM kernel still
  // runs: its tiles then write C = beta C
  DBuf abuf, bbuf, eab, ebb;
  abuf.alloc((size_t)std::max<int64_t>(1, ablk) * tc6::A_BLK, s);
  bbuf.alloc((size_t)std::max<int64_t>(1, g.tc_bblk) * tc6::B_BLK, s);
  eab.alloc(sizeof(int) * std::max<int64_t>(1, nea), s);
  ebb.alloc(sizeof(int) * std::max<int64_t>(1, g.tc_be), s);
  const int sgrid = (int)std::min<int64_t>(items, (int64_t)sms * 16);
  LAUNCH(tc_slice_kernel, sgrid, tc6::SLICE_THREADS, 0, s, g.desc.as<GemmDesc>(), g.tc_dplan.as<TcDescPlan>(),
         g.nprob, g.ntile_tc.as<int2>(), g.tc_eplan.as<TcEntryPlan>(), g.ntilesN_tc, mtL, itemsA, items, b,
         abuf.as<uint8_t>(), eab.as<int>(), bbuf.as<uint8_t>(), ebb.as<int>());
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms);
  LAUNCH(tc_gemm_pre_kernel, grid, tc6::NTHREADS, tc::SMEM, s, g.desc.as<GemmDesc>(), g.tc_dplan.as<TcDescPlan>(),
         g.ntile_tc.as<int2>(), g.tc_eplan.as<TcEntryPlan>(), g.ntilesN_tc, mtiles, mtL, b, abuf.as<uint8_t>(),
         eab.as<int>(), bbuf.as<uint8_t>(), ebb.as<int>());
}

// One column-major GEMM through a batch engine, for the self-check entry
// point: operands are copied (and converted to df64 pairs for engines 1 and
// 2) into stream-ordered work buffers.
void gemm_selftest(int engine, int m, int n, int k, int ta, int tb, double alpha, const double* A, int lda,
                   const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s) {
  const int64_t acols = ta ? m : k, bcols = tb ? k : n;
  DBuf a, bb, c;
  a.alloc(sizeof(double) * std::max<int64_t>(1, (int64_t)lda * acols), s);
  bb.alloc(sizeof(double) * std::max<int64_t>(1, (int64_t)ldb * bcols), s);
  c.alloc(sizeof(double) * std::max<int64_t>(1, (int64_t)ldc * n), s);
  RSF_CUDA(cudaMemcpyAsync(a.p, A, sizeof(double) * lda * acols, cudaMemcpyDeviceToDevice, s));
  RSF_CUDA(cudaMemcpyAsync(bb.p, B, sizeof(double) * ldb * bcols, cudaMemcpyDeviceToDevice, s));
  RSF_CUDA(cudaMemcpyAsync(c.p, C, sizeof(double) * ldc * n, cudaMemcpyDeviceToDevice, s));
  if (engine) {
    convert_df64(a.as<double>(), (int64_t)lda * acols, 1, s);
    convert_df64(bb.as<double>(), (int64_t)ldb * bcols, 1, s);
    convert_df64(c.as<double>(), (int64_t)ldc * n, 1, s);
  }
  GemmDesc d{};
  d.M = m; d.N = n; d.K = k;
  d.lda = lda; d.ldb = ldb; d.ldc = ldc;
  d.a = 0; d.b = 0; d.c = 0;
  d.abase = 0; d.bbase = 1; d.cbase = 2;
  d.ta = (int8_t)ta; d.tb = (int8_t)tb;
  d.alpha = alpha; d.beta = beta;
  GemmBatch g;
  g.build(std::vector<GemmDesc>{d}, s);
  GemmBases b{};
  b.p[0] = a.as<double>(); b.p[1] = bb.as<double>(); b.p[2] = c.as<double>(); b.p[3] = nullptr;
  b.sc[0] = b.sc[1] = b.sc[2] = b.sc[3] = 1;
  b.M = m; b.ld = ldc; b.alpha_scale = 1.0; b.df = engine;
  g.run(b, s);
  if (engine) convert_df64(c.as<double>(), (int64_t)ldc * n, 0, s);
  RSF_CUDA(cudaMemcpyAsync(C, c.p, sizeof(double) * ldc * n, cudaMemcpyDeviceToDevice, s));
  sync(s);
  const int tcs = tc_status_take();
  RSF_CHECK(tcs == 0, (rsf_status)tcs, "tensor-core GEMM: a bounded wait gave up");
}

int tc_status_take() {
  DevStatus h{}, z{};
  RSF_CUDA(cudaMemcpyFromSymbol(&h, g_tc_status, sizeof(DevStatus)));
  if (h.code != 0) RSF_CUDA(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(DevStatus)));
  return h.code;
}

}  // namespace rsf
