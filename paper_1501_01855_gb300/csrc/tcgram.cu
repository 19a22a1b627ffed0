// Gram blocks G[i][j] += (A_i, [gamma5] B_j) on the fifth-generation tensor cores, accurate
// to FP64 level: the dense contractions of the Ritz step (Alg. 6: E = V^dag V,
// M = (V^D)^dag V^D + 2 mu delta V^dag gamma5 V^D) and of the deflated starts (Sec. 4:
// Psi^dag b, (D Psi)^dag b), on FP64 or FP32 fields.
//
// Method: error-free splitting of the operands into small integers (Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast routines of
// matrix multiplication", 2012), with BF16 slices and FP32 accumulation in tensor memory.
// Every vector i gets a power-of-two scale 2^e_i above its largest element; each real
// element x becomes the 42-bit fixed-point integer F = trunc(|x| 2^(42 - e_i)), written in
// six balanced base-128 digits a_1 .. a_6 (a_1 in [0, 128], the others in [-64, 63]), so
// x = sign(x) 2^e_i sum_s a_s 2^(-7 s) up to 2^(e_i - 43) (FP32 operands get the same digits,
// signed, from FP32 arithmetic: tg_digits). Digits are exact in BF16 and
// their products exact in the tensor core; for each group g = s + t (2 .. 8) the products
// a_s b_t summed over 512 reals stay below 2^24 in magnitude, so the FP32 accumulator holds
// that sum exactly. Every 512 reals the seven group sums are read from tensor memory and
// added, scaled by 2^(-7 g), into a double-float (hi + lo FP32) accumulator per output;
// the partial results of the CTAs that split the sum are added in FP64 in a fixed order.
// F is rounded to nearest; the pairs with s + t > 8 (weight 2^-63 and below) are left out.
// The error is then that of representing each operand to 2^(e_i - 43): on Gaussian data
// about 1e-14 of |A_i| |B_j| at 4096 reals and less on longer vectors, the level of an
// FP64 dot product of the same length.
//
// Complex arithmetic: vectors are read as interleaved (re, im) reals. With the A operand
// rows [A_i (64 vectors); A'_i] where A' = (-im, re) per complex element, one MMA of
// M = 128 rows against N = 64 B vectors gives Re (a, b) = sum a.b in rows 0..63 and
// Im (a, b) = sum a'.b in rows 64..127.
//
// One CTA (512 threads) per SM: the operands of the next stage (16 complex elements of 64 A
// and 64 B vectors) are copied into shared memory with cp.async while warps 1..15 slice the
// current one into the canonical no-swizzle K-major layout (core matrices of 8 rows x 16
// bytes), double buffered; thread 0 issues the stage's 52 MMAs (2 K-steps x 26 digit pairs)
// and commits them to the stage's mbarrier, which the slicing of the stage after next waits
// on. Waits are bounded by a 2 s deadline: one that gives up sets the error flag, the CTA
// skips the rest, waits once more (again bounded) for the MMAs it has committed, frees its
// tensor memory and returns, and the host reports OVL_ETIMEOUT.
#include <stdint.h>

#include "kernels.h"

namespace ovl {

namespace {

constexpr int TG_THREADS = 512;
constexpr int TG_S = 6;                          // base-128 digits per real (42 bits)
constexpr int TG_G = 7;                          // groups s + t = 2 .. 8 kept
constexpr int TG_NA = 64;                        // A vectors per tile (M = 128 rows with A')
constexpr int TG_NB = 64;                        // B vectors per tile (N)
constexpr int TG_CPT = TG_NB / (TG_THREADS / 128);   // output columns per thread in the flush
constexpr int TG_KC = 16;                        // complex elements per stage (32 reals)
constexpr int TG_CHUNK = 16;                     // stages per exact accumulation (512 reals)
constexpr int TG_TILE_A = 128 * 32 * 2;          // bytes of one digit tile of A (128 rows x 32 bf16)
constexpr int TG_TILE_B = TG_NB * 32 * 2;        // bytes of one digit tile of B
constexpr int TG_STAGE = TG_S * (TG_TILE_A + TG_TILE_B);
// raw operand staging (cp.async, one stage ahead): 64 A rows then 64 B rows of 16 complex
// elements, rows padded by 16 bytes so that the slicing reads spread over the banks
__host__ __device__ constexpr int tg_esize(int p) { return p == P64 ? 16 : 8; }
__host__ __device__ constexpr int tg_rstride(int p) { return 16 * tg_esize(p) + 16; }
constexpr int TG_RAW = 64 * 2 * tg_rstride(P64);
constexpr int TG_SMEM = 2 * TG_STAGE + 2 * TG_RAW + 1024;   // two digit stages, two raw stages, alignment
constexpr int TG_TMEM_COLS = 512;
static_assert(TG_G * TG_NB <= TG_TMEM_COLS, "group accumulators exceed the tensor-memory allocation");                // 7 groups x 64 columns, rounded to a power of 2
constexpr int TG_EXP_ZERO = -4000;               // scale exponent of an all-zero vector
constexpr unsigned long long TG_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor, K-major without swizzle: start address, leading byte
// offset (distance of core matrices along K), stride byte offset (along the rows), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// true once the barrier's phase with this parity has completed, false after the deadline
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > TG_WAIT_NS) return false;
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// |x| 2^(42 - e) rounded to nearest (ties up), for an IEEE double given by its bits
// (|x| < 2^e, so the result is at most 2^42)
__device__ __forceinline__ unsigned long long fixed_f64(unsigned long long b, int e) {
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0ull;                                  // zero or subnormal: below 2^-1022
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1033 + e - ex;                              // 52 - 42 + e - (ex - 1023) >= 11
  return sh >= 65 ? 0ull : (((m >> (sh - 1)) + 1ull) >> 1);
}

// |x| 2^(42 - e) rounded to nearest (ties up), for an IEEE float given by its bits (|x| < 2^e)
__device__ __forceinline__ unsigned long long fixed_f32(uint32_t b, int e) {
  const int ex = (int)((b >> 23) & 0xFF);
  if (ex == 0) return 0ull;
  const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
  const int t = ex - 108 - e;                                // (ex - 127 - 23) + 42 - e <= 18
  if (t >= 0) return m << t;
  return -t >= 25 ? 0ull : (((m >> (-t - 1)) + 1ull) >> 1);
}

// the loaders give one complex element (from shared memory) as (F_re, F_im) and the sign
// bits of re and im; expo reads the binary exponent of an element in global memory
template <int P>
struct TgLoad;
template <>
struct TgLoad<P64> {
  static __device__ __forceinline__ void get_s(const unsigned char* p, int e, unsigned long long& fr,
                                               unsigned long long& fi, uint32_t& neg) {
    const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(p);
    fr = fixed_f64(w.x, e);
    fi = fixed_f64(w.y, e);
    neg = (uint32_t)(w.x >> 63) | ((uint32_t)(w.y >> 63) << 1);
  }
  static __device__ __forceinline__ int expo(const void* base, size_t q) {
    const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(base) + q);
    return max((int)((w.x >> 52) & 0x7FF), (int)((w.y >> 52) & 0x7FF)) - 1023;
  }
};
template <>
struct TgLoad<P32> {
  static __device__ __forceinline__ void get_s(const unsigned char* p, int e, unsigned long long& fr,
                                               unsigned long long& fi, uint32_t& neg) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    fr = fixed_f32(w.x, e);
    fi = fixed_f32(w.y, e);
    neg = (w.x >> 31) | ((w.y >> 31) << 1);
  }
  static __device__ __forceinline__ int expo(const void* base, size_t q) {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(base) + q);
    return max((int)((w.x >> 23) & 0xFF), (int)((w.y >> 23) & 0xFF)) - 127;
  }
};

// Balanced base-128 digit s (0-based) of the real and the imaginary part, as a BF16 pair
// (real in the low half) with the signs of x applied. g = F + 64 (2^28 + 2^21 + 2^14 + 2^7 +
// 1), F <= 2^42: digit 0 is g >> 35 (0 .. 128), digit s >= 1 is ((g >> (35 - 7 s)) & 127) - 64.
// A digit is placed in the mantissa of 128.0f (bits 16..22; 128 carries into the exponent and
// gives 256), the offset is subtracted exactly, and the upper halves of the two floats are
// the BF16 values (at most 8 significant bits).
__device__ __forceinline__ float tg_digit_f(uint32_t lo, uint32_t hi, int s) {
  if (s == 0) return __uint_as_float(0x43000000u + ((hi >> 3) << 16)) - 128.0f;
  const uint32_t raw = s == 1 ? (__funnelshift_r(lo, hi, 28) & 127u) : ((lo >> (35 - 7 * s)) & 127u);
  return __uint_as_float(0x43000000u | (raw << 16)) - 192.0f;
}
__device__ __forceinline__ uint32_t tg_digit_pair(uint32_t rlo, uint32_t rhi, uint32_t ilo, uint32_t ihi, int s,
                                                  uint32_t negmask) {
  const float fr = tg_digit_f(rlo, rhi, s), fi = tg_digit_f(ilo, ihi, s);
  return __byte_perm(__float_as_uint(fr), __float_as_uint(fi), 0x7632) ^ negmask;
}

constexpr unsigned long long TG_BIAS = 64ull * ((1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

// The six digits of one complex element (from the raw staging buffer) as BF16 pairs,
// negated when neg (gamma5 on B). FP64 operands: the integer splitting above. FP32 operands:
// the same digits by FP32 arithmetic on the FMA pipe, which the integer splitting leaves
// idle: r = x 2^-e (exact, two power-of-two factors), then six times d = round(128 r) by the
// 1.5 x 2^23 addition (exact for |128 r| < 2^22) and r <- 128 r - d (exact: the remainder of
// a float after its nearest integer), so d_0 is in [-128, 128], the others in [-64, 64], and
// |x| 2^-e = sum_s d_s 2^(-7 (s + 1)) up to 2^-43, as for the integer digits (balanced by
// rounding instead of by the bias). A digit is an integer of at most 8 bits, so the upper
// half of its float is its exact BF16.
__device__ __forceinline__ float tg_pow2(int k) { return __int_as_float((127 + k) << 23); }
template <int P>
__device__ __forceinline__ void tg_digits(const unsigned char* p, int e, bool neg, uint32_t pd[TG_S]) {
  if constexpr (P == P32) {
    const float2 w = *reinterpret_cast<const float2*>(p);
    if (e == TG_EXP_ZERO) {
#pragma unroll
      for (int d = 0; d < TG_S; ++d) pd[d] = 0u;
      return;
    }
    const int e1 = e / 2, e2 = e - e1;   // 2^-e as two factors inside the FP32 range
    float rr = __fmul_rn(__fmul_rn(w.x, tg_pow2(-e1)), tg_pow2(-e2));
    float ri = __fmul_rn(__fmul_rn(w.y, tg_pow2(-e1)), tg_pow2(-e2));
    const float M = 12582912.0f;
    const uint32_t nm = neg ? 0x80008000u : 0u;
#pragma unroll
    for (int d = 0; d < TG_S; ++d) {
      const float dr = __fsub_rn(__fmaf_rn(rr, 128.0f, M), M);
      const float di = __fsub_rn(__fmaf_rn(ri, 128.0f, M), M);
      rr = __fmaf_rn(rr, 128.0f, -dr);
      ri = __fmaf_rn(ri, 128.0f, -di);
      pd[d] = __byte_perm(__float_as_uint(dr), __float_as_uint(di), 0x7632) ^ nm;
    }
  } else {
    unsigned long long fr, fi;
    uint32_t sg;
    TgLoad<P>::get_s(p, e, fr, fi, sg);
    if (neg) sg ^= 3u;
    const unsigned long long gr = fr + TG_BIAS, gi = fi + TG_BIAS;
    const uint32_t rlo = (uint32_t)gr, rhi = (uint32_t)(gr >> 32), ilo = (uint32_t)gi, ihi = (uint32_t)(gi >> 32);
    const uint32_t negmask = ((sg & 1u) ? 0x8000u : 0u) | ((sg & 2u) ? 0x80000000u : 0u);
#pragma unroll
    for (int d = 0; d < TG_S; ++d) pd[d] = tg_digit_pair(rlo, rhi, ilo, ihi, d, negmask);
  }
}

// Issue the asynchronous copies of one stage (16 complex elements from q0 of the tile's 64 A
// and 64 B vectors) into a raw staging buffer, 16 bytes per copy, zero-filled past the last
// vector or element; one commit group per call.
template <int PA, int PB>
__device__ __forceinline__ void tg_issue(unsigned char* raw, const void* A, int na, int a0, const void* B, int nb,
                                         int b0, size_t nq, size_t q0, int tid) {
  constexpr int ea = tg_esize(PA), eb = tg_esize(PB);   // bytes per complex element = 16-byte copies per row
  constexpr int sa = tg_rstride(PA), sb = tg_rstride(PB);
  for (int c = tid; c < 64 * (ea + eb); c += TG_THREADS) {
    const bool isA = c < 64 * ea;
    const int cc = isA ? c : c - 64 * ea;
    const int per = isA ? ea : eb;
    const int r = cc / per, k = cc - r * per;
    const size_t qs = q0 + (size_t)(k * 16) / per;       // first complex element of this copy
    const bool ok = isA ? (a0 + r < na) : (b0 + r < nb);
    const bool in = ok && qs < nq;
    const char* src = isA ? reinterpret_cast<const char*>(A) + (size_t)(a0 + (ok ? r : 0)) * nq * ea
                          : reinterpret_cast<const char*>(B) + (size_t)(b0 + (ok ? r : 0)) * nq * eb;
    if (in) src += qs * per;
    const uint32_t dst = smem_u32(raw + (isA ? r * sa : 64 * sa + r * sb) + k * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

}  // namespace

// Per vector: the scale exponent e = 1 + the largest binary exponent of its reals, so that
// every |x| < 2^e (TG_EXP_ZERO for a vector of zeros). One block per vector.
template <int P>
__global__ void __launch_bounds__(256) tc_gram_exp_kernel(const void* X, int n, size_t nq, int* ex) {
  __shared__ int smax;
  if (threadIdx.x == 0) smax = -100000;
  __syncthreads();
  const int i = blockIdx.x;
  const char* base = reinterpret_cast<const char*>(X) + (size_t)i * nq * (P == P64 ? 16 : 8);
  int m = -100000;
  for (size_t q = threadIdx.x; q < nq; q += blockDim.x) m = max(m, TgLoad<P>::expo(base, q));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, m);
  __syncthreads();
  if (threadIdx.x == 0) {
    // a zero or subnormal-only vector reads as the minimum exponent field
    const int lo = P == P64 ? -1023 : -127;
    ex[i] = smax <= lo ? TG_EXP_ZERO : smax + 1;
  }
  (void)n;
}

// grid: (splits of the K range, A tiles x B tiles). partial: per CTA 2 x 64 x 64 doubles
// (Re rows, then Im rows), scaled by 2^(e_i + e_j).
template <int PA, int PB>
__global__ void __launch_bounds__(TG_THREADS, 1)
    tc_gram_kernel(const void* A, int na, const void* B, int nb, size_t nq, int g5q, const int* exa, const int* exb,
                   double* partial, int* err) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ __align__(8) uint64_t fbar;
  __shared__ int abort_flag;
  __shared__ int ea_s[TG_NA], eb_s[TG_NB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x, nsplit = gridDim.x;
  const int ntb = (nb + TG_NB - 1) / TG_NB;
  const int ta = blockIdx.y / ntb, tb = blockIdx.y - ta * ntb;
  const int a0 = ta * TG_NA, b0 = tb * TG_NB;
  const size_t nstage_all = (nq + TG_KC - 1) / TG_KC;
  const size_t st0 = nstage_all * split / nsplit, st1 = nstage_all * (split + 1) / nsplit;
  const int nst = (int)(st1 - st0);

  if (tid < TG_NA) ea_s[tid] = a0 + tid < na ? exa[a0 + tid] : TG_EXP_ZERO;
  else if (tid < TG_NA + TG_NB) eb_s[tid - TG_NA] = b0 + tid - TG_NA < nb ? exb[b0 + tid - TG_NA] : TG_EXP_ZERO;
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TG_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  // instruction descriptor: D F32, A and B BF16, both K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TG_NB >> 3) << 17) | ((128u >> 4) << 24);

  // epilogue ownership: TMEM lane (row) 32 (warp % 4) + lane, columns 16 (warp / 4) .. + 15
  const int row = (warp & 3) * 32 + lane;
  const int cbase = (warp >> 2) * TG_CPT;
  float acc_h[TG_CPT], acc_l[TG_CPT];
#pragma unroll
  for (int c = 0; c < TG_CPT; ++c) acc_h[c] = acc_l[c] = 0.f;

  uint32_t ph = 0u, pend = 0u, fph = 0u;   // bit s: parity / pending commit of stage barrier s
  // slicing tasks of a warp: 8 row groups x 4 K columns for A (tasks 0..31) and for B (32..63)
  const int rl = lane >> 2, kp = lane & 3;
  unsigned char* raw0 = sm + 2 * TG_STAGE;
  if (nst > 0) tg_issue<PA, PB>(raw0, A, na, a0, B, nb, b0, nq, st0 * TG_KC, tid);
  for (int it = 0; it < nst; ++it) {
    const int s = it & 1;
    const int cs = it % TG_CHUNK;   // stage within the exact accumulation chunk
    // the next stage's operands into the other raw buffer (its slicing ended before the
    // barrier that closed the previous iteration); then this stage's own copies
    if (it + 1 < nst)
      tg_issue<PA, PB>(raw0 + ((it + 1) & 1) * TG_RAW, A, na, a0, B, nb, b0, nq, (st0 + it + 1) * TG_KC, tid);
    else
      asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    if ((pend >> s) & 1u) {
      if (mbar_wait(smem_u32(&bar[s]), (ph >> s) & 1u)) {
        ph ^= 1u << s;
        pend &= ~(1u << s);
      } else {
        abort_flag = 1;   // the stage stays pending: the exit waits for it once more
      }
    }
    __syncthreads();
    if (abort_flag) break;
    unsigned char* stA = sm + s * TG_STAGE;
    unsigned char* stB = stA + TG_S * TG_TILE_A;
    const unsigned char* rawA = raw0 + (it & 1) * TG_RAW;
    const unsigned char* rawB = rawA + 64 * tg_rstride(PA);
    const size_t q0 = (st0 + it) * TG_KC;
    // warp 0 issues the MMAs after the barrier: the other warps share the slicing
    for (int task = warp - 1; warp > 0 && task < 64; task += TG_THREADS / 32 - 1) {
      const bool isA = task < 32;
      const int tt = task & 31, rg = tt >> 2, kc = tt & 3;
      const int r = rg * 8 + rl;
      const int j = kc * 4 + kp;
      uint32_t pd[TG_S];   // digit s of (re, im) as a BF16 pair
      if (isA) {
        tg_digits<PA>(rawA + r * tg_rstride(PA) + j * tg_esize(PA), ea_s[r], false, pd);
        // A row r and A' row 64 + r: (re, im) and (-im, re)
        const uint32_t off = (uint32_t)((kc * 16 + rg) * 128 + rl * 16 + kp * 4);
#pragma unroll
        for (int d = 0; d < TG_S; ++d) {
          *reinterpret_cast<uint32_t*>(stA + d * TG_TILE_A + off) = pd[d];
          *reinterpret_cast<uint32_t*>(stA + d * TG_TILE_A + off + 8 * 128) = __byte_perm(pd[d], 0u, 0x1032) ^ 0x8000u;
        }
      } else {
        tg_digits<PB>(rawB + r * tg_rstride(PB) + j * tg_esize(PB), eb_s[r], g5q && q0 + j >= (size_t)g5q, pd);
        const uint32_t off = (uint32_t)((kc * 8 + rg) * 128 + rl * 16 + kp * 4);
#pragma unroll
        for (int d = 0; d < TG_S; ++d) *reinterpret_cast<uint32_t*>(stB + d * TG_TILE_B + off) = pd[d];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const bool chunk_end = (cs == TG_CHUNK - 1) || (it == nst - 1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // descriptors of digit 0, K-step 0 of this stage; the others differ only in the start
      // address (field in the low bits, in units of 16 bytes; no carry out of it below 256 KB)
      const uint64_t da0 = smem_desc(smem_u32(stA), 2048, 128), db0 = smem_desc(smem_u32(stB), 1024, 128);
      const uint32_t acc_chunk = cs > 0 ? 1u : 0u;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {   // two K-steps of 16 reals (2 core-matrix columns each)
#pragma unroll
        for (int g = 0; g < TG_G; ++g) {         // group g + 2 = s + t
#pragma unroll
          for (int ds = (g > TG_S - 1 ? g - TG_S + 1 : 0); ds <= (g < TG_S - 1 ? g : TG_S - 1); ++ds) {
            // digit ds of A, g - ds of B (0-based); the first pair of a group starts its sum
            const uint64_t da = da0 + (uint64_t)((ds * TG_TILE_A + kk * 2 * 2048) >> 4);
            const uint64_t db = db0 + (uint64_t)(((g - ds) * TG_TILE_B + kk * 2 * 1024) >> 4);
            const int first = g > TG_S - 1 ? g - TG_S + 1 : 0;
            mma_bf16(tmem + (uint32_t)(g * TG_NB), da, db, idesc, (kk > 0 || ds > first) ? 1u : acc_chunk);
          }
        }
      }
      mma_commit(smem_u32(&bar[s]));
      if (chunk_end) mma_commit(smem_u32(&fbar));
    }
    pend |= 1u << s;
    if (chunk_end) {
      // the chunk's group sums are exact integers in FP32: add them, scaled, in double-float
      if (!mbar_wait(smem_u32(&fbar), fph)) abort_flag = 1;
      fph ^= 1u;
      __syncthreads();   // abort_flag is read uniformly: tcgen05.ld is warp-collective
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (!abort_flag) {
#pragma unroll
        for (int g = 0; g < TG_G; ++g) {
          uint32_t v[TG_CPT];
          static_assert(TG_CPT == 16, "the flush reads 16 columns per thread");
          const uint32_t ta_ = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * TG_NB + cbase);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15])
              : "r"(ta_));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const float w = __int_as_float((127 - 7 * (g + 2)) << 23);   // 2^(-7 (g + 2))
#pragma unroll
          for (int c = 0; c < TG_CPT; ++c) {
            // TwoSum of acc_h and the exactly scaled group sum
            const float x = __uint_as_float(v[c]) * w;
            const float sum = acc_h[c] + x;
            const float bb = sum - acc_h[c];
            const float e = (acc_h[c] - (sum - bb)) + (x - bb);
            acc_h[c] = sum;
            acc_l[c] += e;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
  }
  // wait for the last commits of each stage barrier before the CTA lets go of its memory,
  // also after an abort (MMAs still in flight must not outlive the tensor memory); each
  // wait again has its own deadline. A commit of a stage also covers every earlier MMA.
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  for (int s = 0; s < 2; ++s)
    if ((pend >> s) & 1u)
      if (!mbar_wait(smem_u32(&bar[s]), (ph >> s) & 1u)) abort_flag = 1;
  __syncthreads();
  if (abort_flag && tid == 0) atomicExch(err, 1);
  if (!abort_flag) {
    const int i = row & 63, reim = row >> 6;
    const int ei = ea_s[i];
    double* out = partial + ((size_t)blockIdx.y * nsplit + split) * 2 * TG_NA * TG_NB + (size_t)reim * TG_NA * TG_NB +
                  (size_t)i * TG_NB;
#pragma unroll
    for (int c = 0; c < TG_CPT; ++c) {
      const int ej = eb_s[cbase + c];
      const double v = (ei == TG_EXP_ZERO || ej == TG_EXP_ZERO) ? 0.0
                                                               : ldexp((double)acc_h[c] + (double)acc_l[c], ei + ej);
      out[cbase + c] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM_COLS));
}

// G[i][j] += sum over the splits (FP64, fixed order)
__global__ void tc_gram_reduce_kernel(const double* partial, int na, int nb, int nsplit, double* G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= na * nb) return;
  const int i = e / nb, j = e - i * nb;
  const int ntb = (nb + TG_NB - 1) / TG_NB;
  const int tile = (i / TG_NA) * ntb + j / TG_NB;
  const int ri = i % TG_NA, cj = j % TG_NB;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    const double* p = partial + ((size_t)tile * nsplit + s) * 2 * TG_NA * TG_NB;
    re += p[(size_t)ri * TG_NB + cj];
    im += p[(size_t)TG_NA * TG_NB + (size_t)ri * TG_NB + cj];
  }
  G[2 * e] += re;
  G[2 * e + 1] += im;
}

bool tc_gram_supported(int pa, int pb) { return (pa == P64 || pa == P32) && (pb == P64 || pb == P32); }

int tc_gram_splits(int na, int nb, int V, int nsm) {
  const int tiles = ((na + TG_NA - 1) / TG_NA) * ((nb + TG_NB - 1) / TG_NB);
  const long long nstage = ((long long)12 * V + TG_KC - 1) / TG_KC;
  long long ns = (nsm + tiles - 1) / tiles;
  const long long maxs = (nstage + TG_CHUNK - 1) / TG_CHUNK;   // at least one chunk per split
  if (ns > maxs) ns = maxs;
  if (ns < 1) ns = 1;
  return (int)ns;
}

size_t tc_gram_work_doubles(int na, int nb, int nsplit) {
  const size_t tiles = (size_t)((na + TG_NA - 1) / TG_NA) * ((nb + TG_NB - 1) / TG_NB);
  return tiles * nsplit * 2 * TG_NA * TG_NB;
}

// A (na vectors), B (nb vectors): fields of precision pa / pb (P64 or P32), 12 V complex
// elements each in the library layout (the element order is the same for both, and
// gamma5 negates the elements from 6 V on). G: na x nb complex FP64 (device), accumulated.
// partial: tc_gram_work_doubles doubles; ex: na + nb ints; err: device int set to 1 when a
// bounded wait gives up.
void launch_tc_gram(int pa, const void* A, int na, int pb, const void* B, int nb, int V, int g5, int nsplit,
                    double* G, double* partial, int* ex, int* err, cudaStream_t st) {
  const size_t nq = (size_t)12 * V;
  int* exa = ex;
  int* exb = ex + na;
  if (pa == P64) tc_gram_exp_kernel<P64><<<na, 256, 0, st>>>(A, na, nq, exa);
  else tc_gram_exp_kernel<P32><<<na, 256, 0, st>>>(A, na, nq, exa);
  if (pb == P64) tc_gram_exp_kernel<P64><<<nb, 256, 0, st>>>(B, nb, nq, exb);
  else tc_gram_exp_kernel<P32><<<nb, 256, 0, st>>>(B, nb, nq, exb);
  const int tiles = ((na + TG_NA - 1) / TG_NA) * ((nb + TG_NB - 1) / TG_NB);
  dim3 grid((unsigned)nsplit, (unsigned)tiles);
  const int g5q = g5 ? (int)(6 * (size_t)V) : 0;
#define TG(X, Y)                                                                                   \
  do {                                                                                             \
    cudaFuncSetAttribute(tc_gram_kernel<X, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, TG_SMEM); \
    tc_gram_kernel<X, Y><<<grid, TG_THREADS, TG_SMEM, st>>>(A, na, B, nb, nq, g5q, exa, exb, partial, err); \
  } while (0)
  if (pa == P64 && pb == P64) TG(P64, P64);
  else if (pa == P32 && pb == P32) TG(P32, P32);
  else if (pa == P64) TG(P64, P32);
  else TG(P32, P64);
#undef TG
  const int nn = na * nb;
  tc_gram_reduce_kernel<<<(nn + 255) / 256, 256, 0, st>>>(partial, na, nb, nsplit, G);
}

}  // namespace ovl
