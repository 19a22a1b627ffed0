// Device-side building blocks of liboverlap: complex arithmetic, the storage
// formats of spinor and link fields, lattice geometry and deterministic block
// reductions.
//
// Device field layouts ("chunked site-major"): a spinor field stores its 12
// complex components (index k = spin*3 + colour) as 16-byte chunks, chunk c of
// site s at [c*V + s], so that a warp reading chunk c of 32 consecutive sites
// issues one fully coalesced 512-byte transaction:
//   F64: 12 chunks of double2 (1 complex)        192 B/site
//   F32:  6 chunks of float4  (2 complex)         96 B/site
//   F16:  3 chunks of 8 halves (4 complex)        48 B/site + one float scale
//         per site (components stored as value / max|component of the site|)
// A batch of n spinors is n such fields back to back.
//
// Links keep only rows 1 and 2 of each SU(3) matrix (12 reals); row 3 is
// rebuilt in registers as conj(row1 x row2). Layout [mu][chunk][V]:
//   F64: 6 chunks double2, F32: 3 chunks float4, F16: 3 chunks of 4 halves.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace ovl {

enum Prec { P64 = 0, P32 = 1, P16 = 2 };

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

// compute type of a storage precision: FP64 storage computes in FP64, the rest in FP32
template <int P> struct Real { using T = float; };
template <> struct Real<P64> { using T = double; };

// ------------------------------------------------------------------ spinors
template <int P> struct SpinorSt;
template <> struct SpinorSt<P64> { static constexpr int NCH = 12; static constexpr int BYTES = 192; };
template <> struct SpinorSt<P32> { static constexpr int NCH = 6; static constexpr int BYTES = 96; };
template <> struct SpinorSt<P16> { static constexpr int NCH = 3; static constexpr int BYTES = 48; };

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

template <int P, typename T, bool RO = false>
struct SpinorLoad;

template <bool RO>
struct SpinorLoad<P64, double, RO> {
  static __device__ __forceinline__ void run(const SpinorRef& f, int rhs, int s, cpx<double> v[12]) {
    const double2* p = reinterpret_cast<const double2*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 w = ldc<RO>(p + (size_t)c * f.V);
      v[c] = cmk(w.x, w.y);
    }
  }
};
template <bool RO>
struct SpinorLoad<P32, float, RO> {
  static __device__ __forceinline__ void run(const SpinorRef& f, int rhs, int s, cpx<float> v[12]) {
    const float4* p = reinterpret_cast<const float4*>(f.data) + (size_t)rhs * 6 * f.V + s;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 w = ldc<RO>(p + (size_t)c * f.V);
      v[2 * c] = cmk(w.x, w.y);
      v[2 * c + 1] = cmk(w.z, w.w);
    }
  }
};
template <bool RO>
struct SpinorLoad<P16, float, RO> {
  static __device__ __forceinline__ void run(const SpinorRef& f, int rhs, int s, cpx<float> v[12]) {
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
};

template <int P, typename T>
__device__ __forceinline__ void load_spinor(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  SpinorLoad<P, T, false>::run(f, rhs, s, v);
}
// read-only path: only for fields that the kernel does not write
template <int P, typename T>
__device__ __forceinline__ void load_spinor_ro(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  SpinorLoad<P, T, true>::run(f, rhs, s, v);
}

template <int P, typename T>
__device__ __forceinline__ void store_spinor(const SpinorRef& f, int rhs, int s, const cpx<T> v[12]);

template <>
__device__ __forceinline__ void store_spinor<P64, double>(const SpinorRef& f, int rhs, int s, const cpx<double> v[12]) {
  double2* p = reinterpret_cast<double2*>(f.data) + (size_t)rhs * 12 * f.V + s;
#pragma unroll
  for (int c = 0; c < 12; ++c) p[(size_t)c * f.V] = make_double2(v[c].r, v[c].i);
}
template <>
__device__ __forceinline__ void store_spinor<P32, float>(const SpinorRef& f, int rhs, int s, const cpx<float> v[12]) {
  float4* p = reinterpret_cast<float4*>(f.data) + (size_t)rhs * 6 * f.V + s;
#pragma unroll
  for (int c = 0; c < 6; ++c) p[(size_t)c * f.V] = make_float4(v[2 * c].r, v[2 * c].i, v[2 * c + 1].r, v[2 * c + 1].i);
}
template <>
__device__ __forceinline__ void store_spinor<P16, float>(const SpinorRef& f, int rhs, int s, const cpx<float> v[12]) {
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

// Store in double, converting to the field's storage.
template <int P>
__device__ __forceinline__ void store_spinor_any(const SpinorRef& f, int rhs, int s, const cpx<double> v[12]) {
  if constexpr (P == P64) {
    store_spinor<P64, double>(f, rhs, s, v);
  } else {
    cpx<float> w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = cmk((float)v[k].r, (float)v[k].i);
    store_spinor<P, float>(f, rhs, s, w);
  }
}
template <int P>
__device__ __forceinline__ void load_spinor_any(const SpinorRef& f, int rhs, int s, cpx<double> v[12]) {
  if constexpr (P == P64) {
    load_spinor<P64, double>(f, rhs, s, v);
  } else {
    cpx<float> w[12];
    load_spinor<P, float>(f, rhs, s, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cmk((double)w[k].r, (double)w[k].i);
  }
}
// Load/store converting between the compute type T and any storage.
template <int P, typename T>
__device__ __forceinline__ void load_spinor_as(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  if constexpr ((P == P64) == (sizeof(T) == 8)) {
    load_spinor<P, T>(f, rhs, s, v);
  } else if constexpr (sizeof(T) == 8) {
    load_spinor_any<P>(f, rhs, s, v);
  } else {
    cpx<double> w[12];
    load_spinor<P64, double>(f, rhs, s, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cmk((float)w[k].r, (float)w[k].i);
  }
}
// read-only variant of load_spinor_as (Wilson-kernel input, never written by that kernel)
template <int P, typename T>
__device__ __forceinline__ void load_spinor_as_ro(const SpinorRef& f, int rhs, int s, cpx<T> v[12]) {
  if constexpr ((P == P64) == (sizeof(T) == 8)) {
    load_spinor_ro<P, T>(f, rhs, s, v);
  } else {
    load_spinor_as<P, T>(f, rhs, s, v);
  }
}

template <int P, typename T>
__device__ __forceinline__ void store_spinor_as(const SpinorRef& f, int rhs, int s, const cpx<T> v[12]) {
  if constexpr ((P == P64) == (sizeof(T) == 8)) {
    store_spinor<P, T>(f, rhs, s, v);
  } else if constexpr (sizeof(T) == 8) {
    store_spinor_any<P>(f, rhs, s, v);
  } else {
    cpx<double> w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = cmk((double)v[k].r, (double)v[k].i);
    store_spinor<P64, double>(f, rhs, s, w);
  }
}

// ------------------------------------------------------------------ links
struct LinkRef {
  const void* data;  // [mu][chunk][V]
  int V;
};

template <typename T>
__device__ __forceinline__ void reconstruct_row3(cpx<T> u[9]) {
  // row3 = conj(row1 x row2)
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

template <int P, typename T>
__device__ __forceinline__ void load_link(const LinkRef& L, int mu, int s, cpx<T> u[9]);

template <>
__device__ __forceinline__ void load_link<P64, double>(const LinkRef& L, int mu, int s, cpx<double> u[9]) {
  const double2* p = reinterpret_cast<const double2*>(L.data) + (size_t)mu * 6 * L.V + s;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double2 w = __ldg(p + (size_t)c * L.V);
    u[c] = cmk(w.x, w.y);
  }
  reconstruct_row3(u);
}
template <>
__device__ __forceinline__ void load_link<P32, float>(const LinkRef& L, int mu, int s, cpx<float> u[9]) {
  const float4* p = reinterpret_cast<const float4*>(L.data) + (size_t)mu * 3 * L.V + s;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 w = __ldg(p + (size_t)c * L.V);
    u[2 * c] = cmk(w.x, w.y);
    u[2 * c + 1] = cmk(w.z, w.w);
  }
  reconstruct_row3(u);
}
template <>
__device__ __forceinline__ void load_link<P16, float>(const LinkRef& L, int mu, int s, cpx<float> u[9]) {
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
  reconstruct_row3(u);
}

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];   // Lx, Ly, Lz, Lt
  int V;
  int bc_t;   // 1: antiperiodic fermion boundary in t
};

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
