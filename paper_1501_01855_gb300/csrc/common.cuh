// Device-side building blocks of liboverlap: complex arithmetic, the double-float
// type, the storage formats of spinor and link fields, lattice geometry and
// deterministic block reductions.
//
// Device field layouts ("chunked site-major"): a spinor field stores its 12
// complex components (index k = spin*3 + colour) as 16-byte chunks, chunk c of
// site s at [c*V + s], so that a warp reading chunk c of 32 consecutive sites
// issues one fully coalesced 512-byte transaction:
//   F64:  12 chunks of double2 (1 complex)                       192 B/site
//   F64E: 12 chunks of float4 (re.hi, re.lo, im.hi, im.lo)        192 B/site
//         = the same number as a double, held as an unevaluated sum hi + lo
//         of two floats (double-float, ~48-bit significand)
//   F32:   6 chunks of float4  (2 complex)                         96 B/site
//   F16:   3 chunks of 8 halves (4 complex)                        48 B/site + one
//         float scale per site (components stored as value / max|component|)
// A batch of n spinors is n such fields back to back.
//
// Links keep only rows 1 and 2 of each SU(3) matrix (12 reals); row 3 is
// rebuilt in registers as conj(row1 x row2). Layout [mu][chunk][V]:
//   F64: 6 chunks double2, F64E: 6 chunks float4, F32: 3 chunks float4,
//   F16: 3 chunks of 4 halves.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace ovl {

enum Prec { P64 = 0, P32 = 1, P16 = 2, P64E = 3 };

// ------------------------------------------------------------------ double-float
// A value hi + lo of two floats with |lo| <= ulp(hi)/2, computed with the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2):
// TwoSum (the exact rounding error of a + b), FastTwoSum (the same when |a| >= |b|)
// and TwoProd via a fused multiply-add (the exact rounding error of a * b). The
// operations below are the "sloppy" double-word sum and product of Hida, Li and
// Bailey (2001, the double-double algorithms of the QD library), done in FP32: a
// relative error of a few units of 2^-47 per operation, every operation on the
// FP32 pipes (GB300 issues FP32 at 60 times its FP64 rate). Intrinsics with explicit
// rounding keep the compiler from contracting or reassociating these sequences.
struct df {
  float hi, lo;
  __host__ __device__ __forceinline__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ __forceinline__ df(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ __forceinline__ df(float x) : hi(x), lo(0.f) {}
  __host__ __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ df(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ bool operator!=(df a, df b) { return a.hi != b.hi || a.lo != b.lo; }

// ------------------------------------------------------------------ complex
template <typename T>
struct cpx {
  T r, i;
};

template <typename T> __host__ __device__ __forceinline__ cpx<T> cmk(T r, T i) { return cpx<T>{r, i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a) { return {-a.r, -a.i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.r, s * a.i}; }
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.r, -a.i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> timesI(cpx<T> a) { return {-a.i, a.r}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> timesMinusI(cpx<T> a) { return {a.i, -a.r}; }
template <typename T> __host__ __device__ __forceinline__ T norm2(cpx<T> a) { return a.r * a.r + a.i * a.i; }

// real-to-double and double-to-compute-type conversions
template <typename T> __device__ __forceinline__ double to_d(T x) { return (double)x; }
template <typename T> __device__ __forceinline__ T from_d(double x) { return (T)x; }
template <> __device__ __forceinline__ df from_d<df>(double x) { return df(x); }

// compute type of a storage precision
template <int P> struct Real { using T = float; };
template <> struct Real<P64> { using T = double; };
template <> struct Real<P64E> { using T = df; };

__host__ __device__ constexpr int spinor_site_bytes(int p) { return p == P32 ? 96 : p == P16 ? 48 : 192; }

// ------------------------------------------------------------------ spinors
// A batch of spinor fields in device memory.
struct SpinorRef {
  void* data;      // 16-byte chunks, [rhs][chunk][V]
  float* norm;     // F16 only: [rhs][V]
  int V;
};

// Chunk load: RO = true goes through the read-only (non-coherent) data path, which
// is only valid for fields that no thread of the same kernel writes; every
// in-place update (x = a x + ..., r -= alpha A p, the SUMR step) uses RO = false,
// otherwise the compiler may legally re-load a value after the kernel's own store.
template <bool RO, typename V>
__device__ __forceinline__ V ldc(const V* p) {
  if constexpr (RO) return __ldg(p);
  else return *p;
}

template <int P, bool RO> struct SpinorIO;

template <bool RO>
struct SpinorIO<P64, RO> {
  static __device__ __forceinline__ void load(const SpinorRef& f, int rhs, int s, cpx<double> v[12]) {
    const double2* p = reinterpret_cast<const double2*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 w = ldc<RO>(p + (size_t)c * f.V);
      v[c] = cmk(w.x, w.y);
    }
  }
  static __device__ __forceinline__ void store(const SpinorRef& f, int rhs, int s, const cpx<double> v[12]) {
    double2* p = reinterpret_cast<double2*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
    for (int c = 0; c < 12; ++c) p[(size_t)c * f.V] = make_double2(v[c].r, v[c].i);
  }
};
template <bool RO>
struct SpinorIO<P64E, RO> {
  static __device__ __forceinline__ void load(const SpinorRef& f, int rhs, int s, cpx<df> v[12]) {
    const float4* p = reinterpret_cast<const float4*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      float4 w = ldc<RO>(p + (size_t)c * f.V);
      v[c] = cmk(df(w.x, w.y), df(w.z, w.w));
    }
  }
  static __device__ __forceinline__ void store(const SpinorRef& f, int rhs, int s, const cpx<df> v[12]) {
    float4* p = reinterpret_cast<float4*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
    for (int c = 0; c < 12; ++c) p[(size_t)c * f.V] = make_float4(v[c].r.hi, v[c].r.lo, v[c].i.hi, v[c].i.lo);
  }
};
template <bool RO>
struct SpinorIO<P32, RO> {
  static __device__ __forceinline__ void load(const SpinorRef& f, int rhs, int s, cpx<float> v[12]) {
    const float4* p = reinterpret_cast<const float4*>(f.data) + (size_t)rhs * 6 * f.V + s;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 w = ldc<RO>(p + (size_t)c * f.V);
      v[2 * c] = cmk(w.x, w.y);
      v[2 * c + 1] = cmk(w.z, w.w);
    }
  }
  static __device__ __forceinline__ void store(const SpinorRef& f, int rhs, int s, const cpx<float> v[12]) {
    float4* p = reinterpret_cast<float4*>(f.data) + (size_t)rhs * 6 * f.V + s;
#pragma unroll
    for (int c = 0; c < 6; ++c) p[(size_t)c * f.V] = make_float4(v[2 * c].r, v[2 * c].i, v[2 * c + 1].r, v[2 * c + 1].i);
  }
};
template <bool RO>
struct SpinorIO<P16, RO> {
  static __device__ __forceinline__ void load(const SpinorRef& f, int rhs, int s, cpx<float> v[12]) {
    const uint4* p = reinterpret_cast<const uint4*>(f.data) + (size_t)rhs * 3 * f.V + s;
    const float sc = ldc<RO>(f.norm + (size_t)rhs * f.V + s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 w = ldc<RO>(p + (size_t)c * f.V);
      const __half2* h = reinterpret_cast<const __half2*>(&w);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 q = __half22float2(h[k]);
        v[4 * c + k] = cmk(q.x * sc, q.y * sc);
      }
    }
  }
  static __device__ __forceinline__ void store(const SpinorRef& f, int rhs, int s, const cpx<float> v[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].r), fabsf(v[k].i)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* p = reinterpret_cast<uint4*>(f.data) + (size_t)rhs * 3 * f.V + s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 w;
      __half2* h = reinterpret_cast<__half2*>(&w);
#pragma unroll
      for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(v[4 * c + k].r * inv, v[4 * c + k].i * inv);
      p[(size_t)c * f.V] = w;
    }
    f.norm[(size_t)rhs * f.V + s] = m;
  }
};

// Loads and stores in any compute type T: the storage's own type directly, anything
// else through double.
template <int P, typename T, bool RO = false>
__device__ __forceinline__ void load_spinor_gen(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  using N = typename Real<P>::T;
  if constexpr (std::is_same<T, N>::value) {
    SpinorIO<P, RO>::load(f, rhs, s, v);
  } else {
    cpx<N> w[12];
    SpinorIO<P, RO>::load(f, rhs, s, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cmk(from_d<T>(to_d(w[k].r)), from_d<T>(to_d(w[k].i)));
  }
}
template <int P, typename T>
__device__ __forceinline__ void store_spinor_gen(const SpinorRef& f, int rhs, int s, const cpx<T> v[12]) {
  using N = typename Real<P>::T;
  if constexpr (std::is_same<T, N>::value) {
    SpinorIO<P, false>::store(f, rhs, s, v);
  } else {
    cpx<N> w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = cmk(from_d<N>(to_d(v[k].r)), from_d<N>(to_d(v[k].i)));
    SpinorIO<P, false>::store(f, rhs, s, w);
  }
}

template <int P, typename T>
__device__ __forceinline__ void load_spinor(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  load_spinor_gen<P, T, false>(f, rhs, s, v);
}
template <int P, typename T>
__device__ __forceinline__ void store_spinor(const SpinorRef& f, int rhs, int s, const cpx<T> v[12]) {
  store_spinor_gen<P, T>(f, rhs, s, v);
}
template <int P, typename T>
__device__ __forceinline__ void load_spinor_as(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  load_spinor_gen<P, T, false>(f, rhs, s, v);
}
// read-only path: only for fields that the kernel does not write (Wilson-kernel input)
template <int P, typename T>
__device__ __forceinline__ void load_spinor_as_ro(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  load_spinor_gen<P, T, true>(f, rhs, s, v);
}
template <int P, typename T>
__device__ __forceinline__ void store_spinor_as(const SpinorRef& f, int rhs, int s, const cpx<T> v[12]) {
  store_spinor_gen<P, T>(f, rhs, s, v);
}
template <int P>
__device__ __forceinline__ void load_spinor_any(const SpinorRef& f, int rhs, int s, cpx<double> v[12]) {
  load_spinor_gen<P, double, false>(f, rhs, s, v);
}
template <int P>
__device__ __forceinline__ void store_spinor_any(const SpinorRef& f, int rhs, int s, const cpx<double> v[12]) {
  store_spinor_gen<P, double>(f, rhs, s, v);
}

// ------------------------------------------------------------------ links
struct LinkRef {
  const void* data;  // [mu][chunk][V]
  int V;
  int variant;       // Wilson-kernel variant chosen for this field (0 thread per site, 1 split)
  int variant_multi; // the variant chosen for launches of 4 or more systems
};

template <typename T>
__device__ __forceinline__ void reconstruct_row3(cpx<T> u[9]) {
  // row3 = conj(row1 x row2)
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

template <int P> struct LinkIO;
template <>
struct LinkIO<P64> {
  static constexpr bool full = false;
  static __device__ __forceinline__ void load(const LinkRef& L, int mu, int s, cpx<double> u[9]) {
    const double2* p = reinterpret_cast<const double2*>(L.data) + (size_t)mu * 6 * L.V + s;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double2 w = __ldg(p + (size_t)c * L.V);
      u[c] = cmk(w.x, w.y);
    }
  }
};
// Double-float links: eight slots per site, one per hop (slot n = 2 mu + b holds U_mu(x)
// for b = 0 and U_mu(x - mu)^dag for b = 1), all 9 entries ([n][9 chunks][V] float4
// chunks). The double-float kernel is bound by FP32 instruction issue, not bytes:
// rebuilding row 3 would cost ~20% of its instructions, and pre-transposed backward
// links let one loop body serve all eight neighbours.
template <>
struct LinkIO<P64E> {
  static constexpr bool full = true;
  static __device__ __forceinline__ void load(const LinkRef& L, int slot, int s, cpx<df> u[9]) {
    const float4* p = reinterpret_cast<const float4*>(L.data) + (size_t)slot * 9 * L.V + s;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float4 w = __ldg(p + (size_t)c * L.V);
      u[c] = cmk(df(w.x, w.y), df(w.z, w.w));
    }
  }
};
template <>
struct LinkIO<P32> {
  static constexpr bool full = false;
  static __device__ __forceinline__ void load(const LinkRef& L, int mu, int s, cpx<float> u[9]) {
    const float4* p = reinterpret_cast<const float4*>(L.data) + (size_t)mu * 3 * L.V + s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 w = __ldg(p + (size_t)c * L.V);
      u[2 * c] = cmk(w.x, w.y);
      u[2 * c + 1] = cmk(w.z, w.w);
    }
  }
};
template <>
struct LinkIO<P16> {
  static constexpr bool full = false;
  static __device__ __forceinline__ void load(const LinkRef& L, int mu, int s, cpx<float> u[9]) {
    const uint2* p = reinterpret_cast<const uint2*>(L.data) + (size_t)mu * 3 * L.V + s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint2 w = __ldg(p + (size_t)c * L.V);
      const __half2* h = reinterpret_cast<const __half2*>(&w);
      float2 a = __half22float2(h[0]);
      float2 b = __half22float2(h[1]);
      u[2 * c] = cmk(a.x, a.y);
      u[2 * c + 1] = cmk(b.x, b.y);
    }
  }
};

template <int P, typename T>
__device__ __forceinline__ void load_link(const LinkRef& L, int mu, int s, cpx<T> u[9]) {
  static_assert(std::is_same<T, typename Real<P>::T>::value, "links load in their own compute type");
  LinkIO<P>::load(L, mu, s, u);
  if constexpr (!LinkIO<P>::full) reconstruct_row3(u);
}

// ------------------------------------------------------------------ geometry
// Site -> coordinates with multiply-shift division (Granlund & Montgomery 1994):
// for n < 2^31 and divisor d, floor(n / d) = (n * m) >> k with k = 31 + ceil(log2 d)
// and m = ceil(2^k / d); exact for every n < 2^31 (m d - 2^k < d <= 2^(k-31)).
struct Geom {
  int L[4];   // Lx, Ly, Lz, Lt
  int V;
  int bc_t;   // 1: antiperiodic fermion boundary in t
  unsigned long long dm[3];   // multipliers for Lx, Ly, Lz
  int dk[3];                  // shifts
};

__device__ __forceinline__ int fdiv(int n, unsigned long long m, int k) {
  return (int)(((unsigned long long)(unsigned)n * m) >> k);
}

__device__ __forceinline__ void site_coords(const Geom& g, int s, int x[4]) {
  int q = fdiv(s, g.dm[0], g.dk[0]);
  x[0] = s - q * g.L[0];
  int q2 = fdiv(q, g.dm[1], g.dk[1]);
  x[1] = q - q2 * g.L[1];
  int q3 = fdiv(q2, g.dm[2], g.dk[2]);
  x[2] = q2 - q3 * g.L[2];
  x[3] = q3;
}

// ------------------------------------------------------------------ reductions
// Sum NV doubles over the x-dimension of a (BX, BY) block, one result per y row,
// in a fixed order (deterministic for a fixed launch shape). Requires BX % 32 == 0.
template <int NV>
__device__ __forceinline__ void block_reduce_rows(double v[NV], double* smem /* BY * (BX/32) * NV */) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) smem[(threadIdx.y * nwarp + warp) * NV + j] = v[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = 0.0;
      for (int w = 0; w < nwarp; ++w) a += smem[(threadIdx.y * nwarp + w) * NV + j];
      v[j] = a;
    }
  }
}

}  // namespace ovl
