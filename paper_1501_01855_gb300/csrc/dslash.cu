// Wilson kernel K of the overlap operator (Sec. 1, the equation for aK_xy):
//
//   K psi(x) = gamma5 [ psi(x) - kappa sum_mu ( (1-gamma_mu) U_mu(x) psi(x+mu)
//                                              + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu) ) ]
//
// One thread per (site, system). (1 -+ gamma_mu) has rank 2, so each neighbour is
// projected to a half spinor (2 spins x 3 colours), multiplied by the link and
// expanded again; the spin algebra below is the DeGrand-Rossi chiral basis,
// gamma5 = diag(1, 1, -1, -1). FP64 / FP32 / FP16 links are 12-real (row 3 rebuilt in
// registers) and the eight neighbours are unrolled; the double-float kernel reads an
// 18-real eight-slot link field and runs one rolled loop over the neighbours (see
// hop_nb_df_core). Threads of one block that share a site but belong to different
// systems read the same links, so the link bytes of a multi-system launch come from L1
// once per block. Launch shapes (chosen per precision by the autotuner at create):
// BX consecutive sites x up to 4 systems per block; four threads per site, one per
// direction; 8x4x4x2 site tiles.
//
// Three fused epilogues cover every use in the sign function (Sec. 3):
//   MODE_K    out = K in, partial sums of ||out||^2 and ||in||^2
//             (first half of a multi-shift CG step: (p, K^2 p) = ||K p||^2);
//   MODE_R    r -= alpha (K t + sigma0 p), partial sums of ||r||^2
//             (second half: K^2 p + sigma0 p applied and consumed in one pass);
//   MODE_OVL  out = c1 v + c2 (y - kappa hop y) = c1 v + c2 gamma5 K y, optionally times
//             gamma5, with partial sums of (w, out): gamma5 eps(K) v and D(mu) v are
//             this with y = sum_i omega_i (K^2 + sigma_i)^-1 v.
// and two for the stored-basis Lanczos form of the same sum (lanczos.cu):
//   MODE_LZK  t = (1 / n_j) K W_j with W_j the system's current basis slot, ||t||^2;
//   MODE_LZL  W_{j+1} = K t - a W_j - b W_{j-1} (the three-term recurrence), ||W_{j+1}||^2.
#include "kernels.h"

namespace ovl {

enum { MODE_K = 0, MODE_R = 1, MODE_OVL = 2, MODE_LZK = 3, MODE_LZL = 4 };

// Register cap per thread, by link precision (and, for FP16 storage, spinor precision).
// Uncapped, the compiler hoists all neighbour loads and takes ~255 registers (8 warps
// per SM): the FP32/FP16 kernels are then latency-bound, and the double-float kernel has
// too few warps to hide its dependent FP32 chains. Swept on 24^3x48 (ms per launch):
//   FP32 K, one system   64: 0.0619 (spills 148 B; the multi-shift r-update form 440 B)
//                        72: 0.0555   80: 0.0557 (best for 12 systems and for a whole FP32 sign)
//                        96: 0.0594
//   FP16 K, one system / 12 systems   72: 0.0575 / 0.5936   80: 0.0578 / 0.5798
//                                     96: 0.0574 / 0.6444  128: 0.0554 / 0.5816
//   double-float K  104: 0.375  112: 0.365  120: 0.438  128: 0.329
// The FP16 cap moves its K launch by 4% at most, and at its best the launch takes as long
// as the FP32 one (0.0553 ms) with half the bytes: the bound is the latency of each site's
// chain of dependent loads, not HBM. FP16 keeps the FP32 cap.
#ifndef OVL_WILSON_REG_DF
#define OVL_WILSON_REG_DF 128
#endif
#ifndef OVL_WILSON_REG_SP
#define OVL_WILSON_REG_SP 80
#endif
#ifndef OVL_WILSON_REG_HP
#define OVL_WILSON_REG_HP OVL_WILSON_REG_SP
#endif
template <int PL, int PIN> struct MaxReg {
  static constexpr int v = PL == P64E ? OVL_WILSON_REG_DF
                         : PL == P64  ? 255
                         : (PL == P16 && PIN == P16) ? OVL_WILSON_REG_HP : OVL_WILSON_REG_SP;
};

// Sums inside the hop term. For double-float operands the sum is "lazy": TwoSum on the
// high words, the low words and the rounding error added in FP32 without the final
// renormalisation. A value hi + lo with |lo| a few ulp(hi) is as good an operand for the
// products below as a normalised one, and the short chains here (at most 8 terms per
// component) keep lo that small; the epilogue's ordinary double-float operations
// renormalise.
template <typename T>
__device__ __forceinline__ cpx<T> padd(cpx<T> a, cpx<T> b) { return a + b; }
__device__ __forceinline__ df lazy_add(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return df(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
template <>
__device__ __forceinline__ cpx<df> padd(cpx<df> a, cpx<df> b) { return {lazy_add(a.r, b.r), lazy_add(a.i, b.i)}; }
template <typename T>
__device__ __forceinline__ cpx<T> psub(cpx<T> a, cpx<T> b) { return padd(a, -b); }

template <int MU, int S, typename T>
__device__ __forceinline__ void project(const cpx<T> p[12], cpx<T> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<T> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if constexpr (MU == 0) {          // h0 = p0 + S i p3, h1 = p1 + S i p2
      h[c] = S > 0 ? padd(p0, timesI(p3)) : psub(p0, timesI(p3));
      h[3 + c] = S > 0 ? padd(p1, timesI(p2)) : psub(p1, timesI(p2));
    } else if constexpr (MU == 1) {   // h0 = p0 - S p3, h1 = p1 + S p2
      h[c] = S > 0 ? psub(p0, p3) : padd(p0, p3);
      h[3 + c] = S > 0 ? padd(p1, p2) : psub(p1, p2);
    } else if constexpr (MU == 2) {   // h0 = p0 + S i p2, h1 = p1 - S i p3
      h[c] = S > 0 ? padd(p0, timesI(p2)) : psub(p0, timesI(p2));
      h[3 + c] = S > 0 ? psub(p1, timesI(p3)) : padd(p1, timesI(p3));
    } else {                          // h0 = p0 + S p2, h1 = p1 + S p3
      h[c] = S > 0 ? padd(p0, p2) : psub(p0, p2);
      h[3 + c] = S > 0 ? padd(p1, p3) : psub(p1, p3);
    }
  }
}

// acc += (1 + S gamma_mu) expanded from the half spinor w
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(cpx<T> acc[12], const cpx<T> w[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<T> w0 = w[c], w1 = w[3 + c];
    acc[c] = padd(acc[c], w0);
    acc[3 + c] = padd(acc[3 + c], w1);
    if constexpr (MU == 0) {          // lower = (-S i w1, -S i w0)
      acc[6 + c] = padd(acc[6 + c], S > 0 ? timesMinusI(w1) : timesI(w1));
      acc[9 + c] = padd(acc[9 + c], S > 0 ? timesMinusI(w0) : timesI(w0));
    } else if constexpr (MU == 1) {   // lower = (S w1, -S w0)
      acc[6 + c] = S > 0 ? padd(acc[6 + c], w1) : psub(acc[6 + c], w1);
      acc[9 + c] = S > 0 ? psub(acc[9 + c], w0) : padd(acc[9 + c], w0);
    } else if constexpr (MU == 2) {   // lower = (-S i w0, S i w1)
      acc[6 + c] = padd(acc[6 + c], S > 0 ? timesMinusI(w0) : timesI(w0));
      acc[9 + c] = padd(acc[9 + c], S > 0 ? timesI(w1) : timesMinusI(w1));
    } else {                          // lower = (S w0, S w1)
      acc[6 + c] = S > 0 ? padd(acc[6 + c], w0) : psub(acc[6 + c], w0);
      acc[9 + c] = S > 0 ? padd(acc[9 + c], w1) : psub(acc[9 + c], w1);
    }
  }
}

template <typename T>
__device__ __forceinline__ void su3_mul(const cpx<T> u[9], const cpx<T> h[6], cpx<T> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      w[3 * sp + a] = u[3 * a] * h[3 * sp] + u[3 * a + 1] * h[3 * sp + 1] + u[3 * a + 2] * h[3 * sp + 2];
}
template <typename T>
__device__ __forceinline__ void su3_dag_mul(const cpx<T> u[9], const cpx<T> h[6], cpx<T> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      w[3 * sp + a] = cmulc(u[a], h[3 * sp]) + cmulc(u[3 + a], h[3 * sp + 1]) + cmulc(u[6 + a], h[3 * sp + 2]);
}

// Double-float link products: every output component is a sum of six real products,
// evaluated as a compensated dot product (Dot2 of Ogita, Rump & Oishi, 2005): the
// high-word products are split exactly by TwoProd (one FMA), summed with TwoSum, and
// every rounding error plus the cross terms hi*lo go to a separate FP32 sum. The
// result (sum, errors) is returned unnormalised; the pair carries about twice FP32
// precision, like the double-float product and sum it replaces, at ~2/3 of the
// instructions.
struct Dot2 {
  float s, c;
};
__device__ __forceinline__ Dot2 dot2_first(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return {p, e};
}
__device__ __forceinline__ void dot2_add(Dot2& a, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(a.s, p);
  const float v = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, v)), __fsub_rn(p, v));
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}
// w = U h: re = sum_b (Ur hr - Ui hi), im = sum_b (Ur hi + Ui hr)
__device__ __forceinline__ void su3_mul(const cpx<df> u[9], const cpx<df> h[6], cpx<df> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cpx<df>* r = u + 3 * a;
      const cpx<df>* v = h + 3 * sp;
      Dot2 re = dot2_first(r[0].r, v[0].r), im = dot2_first(r[0].r, v[0].i);
      dot2_add(re, -r[0].i, v[0].i);
      dot2_add(im, r[0].i, v[0].r);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        dot2_add(re, r[b].r, v[b].r);
        dot2_add(re, -r[b].i, v[b].i);
        dot2_add(im, r[b].r, v[b].i);
        dot2_add(im, r[b].i, v[b].r);
      }
      w[3 * sp + a] = cmk(df(re.s, re.c), df(im.s, im.c));
    }
}
// w = U^dag h: re = sum_b (Ur hr + Ui hi), im = sum_b (Ur hi - Ui hr), U = U[b][a]
__device__ __forceinline__ void su3_dag_mul(const cpx<df> u[9], const cpx<df> h[6], cpx<df> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cpx<df>* v = h + 3 * sp;
      Dot2 re = dot2_first(u[a].r, v[0].r), im = dot2_first(u[a].r, v[0].i);
      dot2_add(re, u[a].i, v[0].i);
      dot2_add(im, -u[a].i, v[0].r);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        dot2_add(re, u[3 * b + a].r, v[b].r);
        dot2_add(re, u[3 * b + a].i, v[b].i);
        dot2_add(im, u[3 * b + a].r, v[b].i);
        dot2_add(im, -u[3 * b + a].i, v[b].r);
      }
      w[3 * sp + a] = cmk(df(re.s, re.c), df(im.s, im.c));
    }
}

// Per-thread sums for the epilogue reductions, kept in the compute type: GB300 runs
// FP64 (and FP32 <-> FP64 conversions) at a small fraction of its FP32 rate, so the FP32
// and FP16-storage kernels sum in FP32 (their own precision) and convert once; the
// double-float kernel sums with Dot2, which keeps its FP64-level accuracy on FP32 pipes.
template <typename T> struct RedT { using type = double; };
template <> struct RedT<float> { using type = float; };
template <typename T> struct Acc {
  T s = T(0);
  __device__ __forceinline__ void add(T x, T y) { s = fma(x, y, s); }
  __device__ __forceinline__ typename RedT<T>::type get() const { return s; }
};
template <> struct Acc<df> {
  Dot2 d = {0.f, 0.f};
  __device__ __forceinline__ void add(df x, df y) { dot2_add(d, x, y); }
  __device__ __forceinline__ double get() const { return (double)d.s + (double)d.c; }
};
template <typename T>
__device__ __forceinline__ void acc_norm(Acc<T>& a, const cpx<T>& z) {
  a.add(z.r, z.r);
  a.add(z.i, z.i);
}

// ---- double-float hop: one rolled loop over the eight neighbours -------------------
// The double-float kernel issues ~1k FP32 instructions per neighbour; unrolled over all
// eight it is too large for the instruction cache (ncu: "no instruction" was the top
// stall). Here one loop body serves every neighbour n = 2 mu + b (b = 0 forward, 1
// backward): the spin structure of (1 -+ gamma_mu) is the same for all eight up to
// which lower spin pairs with which upper one and a power of i, and the link of hop n
// is read from slot n of the eight-slot link field (U_mu(x), or U_mu(x - mu)^dag with
// the boundary sign folded in), so the product is always U h.

// i^k z, exact (a swap and sign changes), for a runtime k
__device__ __forceinline__ cpx<df> ipow(const cpx<df>& z, int k) {
  const bool odd = (k & 1) != 0;
  const df re = odd ? z.i : z.r;
  const df im = odd ? z.r : z.i;
  const float sr = (k == 1 || k == 2) ? -1.f : 1.f;
  const float si = k >= 2 ? -1.f : 1.f;
  return {df(__fmul_rn(re.hi, sr), __fmul_rn(re.lo, sr)), df(__fmul_rn(im.hi, si), __fmul_rn(im.lo, si))};
}

// site of neighbour n = 2 mu + b of site s (coordinates x), periodic wrap
__device__ __forceinline__ int nb_site(const Geom& g, const int x[4], int s, int n) {
  const int mu = n >> 1;
  const bool fwd = (n & 1) == 0;
  const int xm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
  const int lm = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
  const int st = mu == 0 ? 1 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
  return fwd ? (xm == lm - 1 ? s - (lm - 1) * st : s + st) : (xm == 0 ? s + (lm - 1) * st : s - st);
}

// hop n given the neighbour spinor psi: acc += (1 -+ gamma_mu) W_n(s) psi
__device__ __forceinline__ void hop_nb_df_core(const LinkRef& L, int s, int n, const cpx<df> psi[12],
                                               cpx<df> acc[12]) {
  const int mu = n >> 1;
  const bool fwd = (n & 1) == 0;
  // In powers of i, with S = -1 (forward) or +1 (backward) = i^sS:
  //   h0 = psi0 + i^a0 psi_j0,  h1 = psi1 + i^a1 psi_(5-j0)
  //   lower spins of (1 + S gamma_mu) w: acc2 += i^b0 w_k0, acc3 += i^b1 w_(1-k0)
  // mu = 0: j0 3, a0 a1 sS+1, k0 1, b0 b1 sS+3;  mu = 1: j0 3, a0 sS+2, a1 sS, k0 1, b0 sS, b1 sS+2
  // mu = 2: j0 2, a0 sS+1, a1 sS+3, k0 0, b0 sS+3, b1 sS+1;  mu = 3: j0 2, a0 a1 b0 b1 sS, k0 0
  const int sS = fwd ? 2 : 0;
  const bool lo3 = mu <= 1;   // j0 = 3 and k0 = 1
  const int a0 = (sS + (mu == 0 || mu == 2 ? 1 : mu == 1 ? 2 : 0)) & 3;
  const int a1 = (sS + (mu == 0 ? 1 : mu == 2 ? 3 : 0)) & 3;
  const int b0 = (sS + (mu == 0 || mu == 2 ? 3 : 0)) & 3;
  const int b1 = (sS + (mu == 0 ? 3 : mu == 1 ? 2 : mu == 2 ? 1 : 0)) & 3;
  cpx<df> h[6], w[6], u[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<df> pa = lo3 ? psi[9 + c] : psi[6 + c];
    const cpx<df> pb = lo3 ? psi[6 + c] : psi[9 + c];
    h[c] = padd(psi[c], ipow(pa, a0));
    h[3 + c] = padd(psi[3 + c], ipow(pb, a1));
  }
  LinkIO<P64E>::load(L, n, s, u);
  su3_mul(u, h, w);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = padd(acc[c], w[c]);
    acc[3 + c] = padd(acc[3 + c], w[3 + c]);
    const cpx<df> wa = lo3 ? w[3 + c] : w[c];
    const cpx<df> wb = lo3 ? w[c] : w[3 + c];
    acc[6 + c] = padd(acc[6 + c], ipow(wa, b0));
    acc[9 + c] = padd(acc[9 + c], ipow(wb, b1));
  }
}

template <int PIN>
__device__ __forceinline__ void hop_nb_df(const Geom& g, const LinkRef& L, const SpinorRef& in, int rhs, int s,
                                          const int x[4], int n, cpx<df> acc[12]) {
  cpx<df> psi[12];
  load_spinor_as_ro<PIN, df>(in, rhs, nb_site(g, x, s, n), psi);
  hop_nb_df_core(L, s, n, psi, acc);
}

template <int MU, int PIN, int PL, typename T>
__device__ __forceinline__ void hop_dir(const Geom& g, const LinkRef& L, const SpinorRef& in, int rhs, int s,
                                        const int x[4], int stride, cpx<T> acc[12]) {
  if constexpr (PL == P64E) {
    hop_nb_df<PIN>(g, L, in, rhs, s, x, 2 * MU, acc);
    hop_nb_df<PIN>(g, L, in, rhs, s, x, 2 * MU + 1, acc);
    return;
  } else {
  cpx<T> psi[12], h[6], w[6], u[9];
  // forward neighbour: (1 - gamma_mu) U_mu(x) psi(x + mu)
  {
    const bool wrap = x[MU] == g.L[MU] - 1;
    const int sf = wrap ? s - (g.L[MU] - 1) * stride : s + stride;
    load_spinor_as_ro<PIN, T>(in, rhs, sf, psi);
    project<MU, -1>(psi, h);
    if (MU == 3 && g.bc_t && wrap) {
#pragma unroll
      for (int k = 0; k < 6; ++k) h[k] = -h[k];
    }
    load_link<PL, T>(L, MU, s, u);
    su3_mul(u, h, w);
    accumulate<MU, -1>(acc, w);
  }
  // backward neighbour: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
  {
    const bool wrap = x[MU] == 0;
    const int sb = wrap ? s + (g.L[MU] - 1) * stride : s - stride;
    load_spinor_as_ro<PIN, T>(in, rhs, sb, psi);
    project<MU, +1>(psi, h);
    if (MU == 3 && g.bc_t && wrap) {
#pragma unroll
      for (int k = 0; k < 6; ++k) h[k] = -h[k];
    }
    load_link<PL, T>(L, MU, sb, u);
    su3_dag_mul(u, h, w);
    accumulate<MU, +1>(acc, w);
  }
  }
}

// Prefetch into L1 the lines hop n of the double-float loop reads: the neighbour's
// twelve spinor chunks and the nine link entries of slot n. Issued one hop ahead, so that
// the loads of the next hop find their lines in L1 instead of waiting on L2; it holds no
// registers.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
template <int PIN>
__device__ __forceinline__ void prefetch_hop_df(const Geom& g, const LinkRef& L, const SpinorRef& in, int rhs,
                                                int s, const int x[4], int n) {
  if constexpr (PIN == P64E) {
    const float4* p = reinterpret_cast<const float4*>(in.data) + (size_t)rhs * 12 * in.V + nb_site(g, x, s, n);
#pragma unroll
    for (int c = 0; c < 12; ++c) prefetch_l1(p + (size_t)c * in.V);
  }
  const float4* q = reinterpret_cast<const float4*>(L.data) + (size_t)n * 9 * L.V + s;
#pragma unroll
  for (int c = 0; c < 9; ++c) prefetch_l1(q + (size_t)c * L.V);
}

#ifndef OVL_DF_PREFETCH
#define OVL_DF_PREFETCH 1
#endif
template <int PIN, int PL, typename T>
__device__ __forceinline__ void hop(const Geom& g, const LinkRef& L, const SpinorRef& in, int rhs, int s,
                                    const int x[4], cpx<T> acc[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cmk(T(0), T(0));
  if constexpr (PL == P64E) {
    if (OVL_DF_PREFETCH) prefetch_hop_df<PIN>(g, L, in, rhs, s, x, 0);
#pragma unroll 1
    for (int n = 0; n < 8; ++n) {
      if (OVL_DF_PREFETCH && n < 7) prefetch_hop_df<PIN>(g, L, in, rhs, s, x, n + 1);
      hop_nb_df<PIN>(g, L, in, rhs, s, x, n, acc);
    }
    return;
  }
  const int sy = g.L[0], sz = g.L[0] * g.L[1], st = sz * g.L[2];
  hop_dir<0, PIN, PL, T>(g, L, in, rhs, s, x, 1, acc);
  hop_dir<1, PIN, PL, T>(g, L, in, rhs, s, x, sy, acc);
  hop_dir<2, PIN, PL, T>(g, L, in, rhs, s, x, sz, acc);
  hop_dir<3, PIN, PL, T>(g, L, in, rhs, s, x, st, acc);
}

struct DArgs {
  Geom g;
  double kappa;
  LinkRef links;
  SpinorRef in, out, aux1, aux2;
  int nrhs, nsb, ngr;
  double* partials;
  const MsRhs* ms;
  double sigma0;
  double c1, c2;
  const double* coef;
  int herm;
  int variant;   // 0: thread per site, 1: direction split, 2: 4D tiles, 3: lane pairs
  LzRhs* lz;
  LzCtl lzc;
};

// ---- the scalar step of the stored-basis Lanczos, fused into its Wilson launches -------
// Called by the whole block for a system whose last partial sum this block wrote. The
// sum over the site-block partials runs in a fixed order (thread-strided, then a fixed
// tree), so the result does not depend on which block came last.
__device__ __forceinline__ double lz_block_sum(const double* partials, int nsb, int rhs, double* sm) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  // eight loads in flight per thread (a block of 64 threads sums 2048 partials of a 16^3 x 32
  // lattice: one dependent L2 load after another would hold the launch for microseconds);
  // the eight running sums are combined in a fixed order
  const double* base = partials + (size_t)rhs * nsb * NVRED;
  double acc8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int b = tid;
  for (; b + 7 * nt < nsb; b += 8 * nt) {
#pragma unroll
    for (int u = 0; u < 8; ++u) acc8[u] += __ldcg(base + (size_t)(b + u * nt) * NVRED);
  }
  for (int u = 0; b < nsb; b += nt, ++u) acc8[u & 7] += __ldcg(base + (size_t)b * NVRED);
  const double v = ((acc8[0] + acc8[1]) + (acc8[2] + acc8[3])) + ((acc8[4] + acc8[5]) + (acc8[6] + acc8[7]));
  sm[tid] = v;
  for (int i = nt + tid; i < 256; i += nt) sm[i] = 0.0;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) sm[tid] += sm[tid + o];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

template <int MODE>
__device__ void lz_finish(const DArgs& a, int rhs) {
  __shared__ double sm[256], em[256];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  LzRhs& L = a.lz[rhs];
  const bool skip = L.done != 0;   // read by every thread before any write below
  __syncthreads();
  if (!skip) {
    const double tot = lz_block_sum(a.partials, a.nsb, rhs, sm);
    if constexpr (MODE == MODE_LZK) {
      if (tid == 0) {
        a.lzc.ahist[(size_t)rhs * a.lzc.hcap + L.j] = tot;
        L.alpha = tot;
        L.a = tot * L.inv_n;
        L.b = L.j > 0 ? L.beta_prev * L.inv_nprev : 0.0;
        if (!(tot > 0.0) || !isfinite(tot)) {
          L.done = 1;
          L.status = 2;   // K^2 is positive definite: breakdown
          L.finished = 1;
        }
      }
    } else {
      const Poles* P = a.lzc.poles;
      const double beta = sqrt(tot);
      const int j = L.j;
      const double alpha = L.alpha, bp = L.beta_prev;
      double e = 0.0, m = 0.0;
      for (int i = tid; i < P->n; i += nt) {
        const double sg = P->sigma0 + P->ds[i];
        const double d = alpha + sg - (j > 0 ? bp * bp / L.d[i] : 0.0);
        L.d[i] = d;
        L.rho[i] *= beta / d;
        const double ei = fabs(L.w[i]) * P->gbound[i] * L.rho[i];
        e += ei;
        m = fmax(m, ei);
      }
      sm[tid] = e;
      em[tid] = m;
      for (int i = nt + tid; i < 256; i += nt) sm[i] = em[i] = 0.0;
      __syncthreads();
      for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
          sm[tid] += sm[tid + o];
          em[tid] = fmax(em[tid], em[tid + o]);
        }
        __syncthreads();
      }
      if (tid == 0) {
        a.lzc.bhist[(size_t)rhs * a.lzc.hcap + j] = beta;
        L.err = sm[0];
        L.total += 1;
        L.w_reads += (j > 0 ? 2 : 1);
        L.inv_nprev = L.inv_n;
        L.inv_n = beta > 0.0 ? 1.0 / beta : 0.0;
        L.beta_prev = beta;
        L.j = j + 1;
        if (!isfinite(beta) || !isfinite(sm[0])) {
          L.done = 1;
          L.status = 2;
          L.finished = 1;
        } else if ((L.even ? em[0] * P->n <= L.thr : sm[0] <= L.thr) || beta == 0.0) {
          // within budget, or an invariant subspace (the Galerkin solutions are exact)
          L.done = 1;
          L.status = 0;
          L.finished = 1;
        } else if (L.total >= L.maxit) {
          L.done = 1;
          L.status = 1;
          L.finished = 1;
        } else if (L.j + 1 > L.cap - 1) {
          L.done = 1;
          L.status = 3;   // W_{j+2} would not fit: restart from W_{j+1}
        }
      }
    }
  }
  if (tid == 0) a.lzc.ctr[rhs] = 0u;
  __syncthreads();
}

// After the block's partial sums are written (by thread x = 0 of each row y, for system
// rhs_y): count the block in, and finish every system for which it came last. nblk: blocks
// that write partials for one system. Every thread of the block calls this.
template <int MODE>
__device__ __forceinline__ void lz_arrive(const DArgs& a, int rhs_row, int nblk) {
  __shared__ int last[8], rows[8];
  if (threadIdx.x == 0) {
    int f = 0;
    if (rhs_row < a.nrhs) {
      __threadfence();   // this row's partial sum before the count
      f = atomicAdd(&a.lzc.ctr[rhs_row], 1u) == (unsigned)(nblk - 1) ? 1 : 0;
    }
    last[threadIdx.y] = f;
    rows[threadIdx.y] = rhs_row;
  }
  __syncthreads();
  for (int y = 0; y < (int)blockDim.y; ++y) {
    if (last[y]) {   // shared, so the same for every thread of the block
      __threadfence();
      lz_finish<MODE>(a, rows[y]);
    }
  }
}

// Epilogue shared by both kernel variants: acc holds the hop sum of site s; v gets this
// thread's contributions to the NVRED partial sums (see the mode list at the top).
template <int MODE, int PIN, int POUT, int PA1, int PA2, typename T>
__device__ __forceinline__ void wilson_epilogue(const DArgs& a, int rhs, int fin, int s, cpx<T> acc[12],
                                                typename RedT<T>::type v[NVRED]) {
  cpx<T> c[12];
  load_spinor_as_ro<PIN, T>(a.in, fin, s, c);
  const T kap = (T)a.kappa;
  const bool red = a.partials != nullptr;
  if constexpr (MODE == MODE_LZK) {
    // t = (1 / n_j) gamma5 (W_j - kappa hop W_j)
    const T sc = (T)a.lz[rhs].inv_n;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cpx<T> o = c[k] - kap * acc[k];
      if (k >= 6) o = -o;
      acc[k] = sc * o;
    }
    store_spinor_as<POUT, T>(a.out, rhs, s, acc);
    if (red) {
      Acc<T> n0;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc_norm(n0, acc[k]);
      v[0] = n0.get();
    }
  } else if constexpr (MODE == MODE_LZL) {
    // W_{j+1} = gamma5 (t - kappa hop t) - a W_j - b W_{j-1}
    const LzRhs& L = a.lz[rhs];
    const int j = L.j;
    const T ca = (T)L.a, cb = (T)L.b;
    cpx<T> w[12];
    load_spinor_as<PA1, T>(a.aux1, j * a.nrhs + rhs, s, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cpx<T> o = c[k] - kap * acc[k];
      if (k >= 6) o = -o;
      acc[k] = o - ca * w[k];
    }
    if (j > 0) {
      load_spinor_as<PA1, T>(a.aux1, (j - 1) * a.nrhs + rhs, s, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = acc[k] - cb * w[k];
    }
    store_spinor_as<POUT, T>(a.out, (j + 1) * a.nrhs + rhs, s, acc);
    if (red) {
      Acc<T> n0;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc_norm(n0, acc[k]);
      v[0] = n0.get();
    }
  } else if constexpr (MODE == MODE_K) {
    // K in = gamma5 (in - kappa acc)
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cpx<T> o = c[k] - kap * acc[k];
      if (k >= 6) o = -o;
      acc[k] = o;
    }
    store_spinor_as<POUT, T>(a.out, rhs, s, acc);
    if (red) {
      Acc<T> n0, n1;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        acc_norm(n0, acc[k]);
        acc_norm(n1, c[k]);
      }
      v[0] = n0.get();
      v[1] = n1.get();
    }
  } else if constexpr (MODE == MODE_R) {
    cpx<T> p[12], r[12];
    load_spinor_as<PA1, T>(a.aux1, rhs, s, p);
    load_spinor_as<PA2, T>(a.aux2, rhs, s, r);
    const T sg = (T)a.sigma0;
    const T al = (T)a.ms[rhs].alpha;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cpx<T> o = c[k] - kap * acc[k];
      if (k >= 6) o = -o;
      o = o + sg * p[k];
      r[k] = r[k] - al * o;
    }
    store_spinor_as<PA2, T>(a.aux2, rhs, s, r);
    if (red) {
      Acc<T> n0;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc_norm(n0, r[k]);
      v[0] = n0.get();
    }
  } else {
    cpx<T> w[12];
    T c1 = (T)a.c1, c2 = (T)a.c2;
    if (a.coef != nullptr) {
      c1 = (T)a.coef[2 * rhs];
      c2 = (T)a.coef[2 * rhs + 1];
    }
    if (c1 != T(0)) {
      load_spinor_as<PA1, T>(a.aux1, rhs, s, w);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) w[k] = cmk(T(0), T(0));
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cpx<T> o = c1 * w[k] + c2 * (c[k] - kap * acc[k]);
      if (a.herm && k >= 6) o = -o;
      acc[k] = o;
    }
    store_spinor_as<POUT, T>(a.out, rhs, s, acc);
    if (red) {
      load_spinor_as<PA2, T>(a.aux2, rhs, s, w);
      Acc<T> dr, di, n0, n1;   // (w, out) = sum conj(w) out
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        dr.add(w[k].r, acc[k].r);
        dr.add(w[k].i, acc[k].i);
        di.add(w[k].r, acc[k].i);
        di.add(-w[k].i, acc[k].r);
        acc_norm(n0, acc[k]);
        acc_norm(n1, w[k]);
      }
      v[0] = dr.get();
      v[1] = di.get();
      v[2] = n0.get();
      v[3] = n1.get();
    }
  }
}

// Block sum of the per-thread partials: warp stage in R (FP32 for the FP32 kernels),
// then FP64 across warps in a fixed order; the result is valid on thread (0, y).
template <typename R>
__device__ __forceinline__ void block_reduce_partials(R v[NVRED], double* smem, double out[NVRED]) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NVRED; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NVRED; ++j) smem[(threadIdx.y * nwarp + warp) * NVRED + j] = (double)v[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NVRED; ++j) {
      double t = 0.0;
      for (int w = 0; w < nwarp; ++w) t += smem[(threadIdx.y * nwarp + w) * NVRED + j];
      out[j] = t;
    }
  }
}

// Variant 0: one thread per (site, system) walks all eight neighbours; a block is BX
// consecutive sites (x fastest) times up to 4 systems.
// Variant 2 (TILED): a block is one system on a 4D tile of TX x TY x TZ x TT = 256 sites,
// so that the neighbours in all four directions mostly lie in the block's own tile
// (L1 hits) instead of BX/Lx rows away in z and t. Needs every extent divisible by the
// tile. Its block sum goes to the first of the tile's 256/BX partial slots (the others
// get zero), so the partial layout (system, BX-site block) is the same for all variants.
constexpr int TX = 8, TY = 4, TZ = 4, TT = 2;
template <int MODE, int PIN, int PL, int POUT, int PA1, int PA2, bool TILED>
__global__ void __launch_bounds__(256) __maxnreg__((MaxReg<PL, PIN>::v)) wilson_kernel(const DArgs a) {
  using T = typename Real<PL>::T;
  __shared__ double red[4 * (BX / 32) * NVRED];
  int sb, rhs, s;
  int x[4];
  bool live;
  if constexpr (TILED) {
    const int ntx = a.g.L[0] / TX, nty = a.g.L[1] / TY, ntz = a.g.L[2] / TZ;
    int b = blockIdx.x;
    const int bx = b % ntx;
    b /= ntx;
    const int by = b % nty;
    b /= nty;
    const int bz = b % ntz;
    const int bt = b / ntz;
    const int t = threadIdx.x;
    x[0] = bx * TX + (t & 7);
    x[1] = by * TY + ((t >> 3) & 3);
    x[2] = bz * TZ + ((t >> 5) & 3);
    x[3] = bt * TT + (t >> 7);
    s = ((x[3] * a.g.L[2] + x[2]) * a.g.L[1] + x[1]) * a.g.L[0] + x[0];
    rhs = blockIdx.y;
    sb = blockIdx.x * (TX * TY * TZ * TT / BX);
    live = rhs < a.nrhs;
  } else {
    sb = blockIdx.x / a.ngr;
    const int rg = blockIdx.x - sb * a.ngr;
    rhs = rg * blockDim.y + threadIdx.y;
    s = sb * BX + threadIdx.x;
    live = (s < a.g.V) && (rhs < a.nrhs);
    if (live) site_coords(a.g, s, x);
  }
  if (live && a.ms != nullptr && (MODE == MODE_K || MODE == MODE_R)) live = !a.ms[rhs].done;
  int fin = rhs;   // field index of the hop input (the basis slot in MODE_LZK)
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (live) live = !a.lz[rhs].done;
    if (MODE == MODE_LZK && live) fin = a.lz[rhs].j * a.nrhs + rhs;
  }
  using R = typename RedT<T>::type;
  R v[NVRED] = {R(0), R(0), R(0), R(0)};
  if (live) {
    cpx<T> acc[12];
    hop<PIN, PL, T>(a.g, a.links, a.in, fin, s, x, acc);
    wilson_epilogue<MODE, PIN, POUT, PA1, PA2, T>(a, rhs, fin, s, acc, v);
  }
  if (a.partials != nullptr) {
    double tot[NVRED];
    block_reduce_partials<R>(v, red, tot);
    if (threadIdx.x == 0 && rhs < a.nrhs) {
#pragma unroll
      for (int j = 0; j < NVRED; ++j) a.partials[((size_t)rhs * a.nsb + sb) * NVRED + j] = tot[j];
      if constexpr (TILED) {
        for (int q = 1; q < TX * TY * TZ * TT / BX; ++q)
#pragma unroll
          for (int j = 0; j < NVRED; ++j) a.partials[((size_t)rhs * a.nsb + sb + q) * NVRED + j] = 0.0;
      }
    }
  }
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (a.lzc.ctr != nullptr) lz_arrive<MODE>(a, rhs, TILED ? (int)gridDim.x : a.nsb);
  }
}

// ---- variant 3 (double-float only): two threads per (site, system) ----------------------
// The projection (1 -+ gamma_mu) leaves two half spinors h0, h1 (upper spins 0 and 1 plus a
// power of i times a lower spin); thread `half` of a lane pair builds h_half, multiplies it
// by the link (U h_half, row by row) and adds the result to upper spin `half` and to one
// lower spin, which for mu <= 1 is spin 3 - half and for mu >= 2 spin 2 + half. So each
// thread holds three accumulators (upper spin, lower spin from mu <= 1, from mu >= 2); at
// the end one shuffle between the pair completes the lower spins, and thread `half` owns
// output spins half and 2 + half. No arithmetic is duplicated: the pair does the work of
// one thread of variant 0 with about two thirds of the registers each, so more warps hide
// the load latency; the two lanes of a pair read the same link entries (one broadcast).
__device__ __forceinline__ cpx<df> ld_cdf(const SpinorRef& f, int fld, int s, int k) {
  const float4 w = *(reinterpret_cast<const float4*>(f.data) + ((size_t)fld * 12 + k) * f.V + s);
  return cmk(df(w.x, w.y), df(w.z, w.w));
}
__device__ __forceinline__ cpx<df> ldg_cdf(const SpinorRef& f, int fld, int s, int k) {
  const float4 w = __ldg(reinterpret_cast<const float4*>(f.data) + ((size_t)fld * 12 + k) * f.V + s);
  return cmk(df(w.x, w.y), df(w.z, w.w));
}
__device__ __forceinline__ void st_cdf(const SpinorRef& f, int fld, int s, int k, const cpx<df>& v) {
  *(reinterpret_cast<float4*>(f.data) + ((size_t)fld * 12 + k) * f.V + s) =
      make_float4(v.r.hi, v.r.lo, v.i.hi, v.i.lo);
}
__device__ __forceinline__ cpx<df> shfl_pair(const cpx<df>& v) {
  return cmk(df(__shfl_xor_sync(0xffffffffu, v.r.hi, 1), __shfl_xor_sync(0xffffffffu, v.r.lo, 1)),
             df(__shfl_xor_sync(0xffffffffu, v.i.hi, 1), __shfl_xor_sync(0xffffffffu, v.i.lo, 1)));
}

// acc6 (components 3 half + c and 3 (2 + half) + c of site s) through the epilogue of MODE;
// v receives this thread's share of the partial sums.
template <int MODE>
__device__ __forceinline__ void pair_epilogue(const DArgs& a, int rhs, int fin, int s, int half, cpx<df> acc6[6],
                                              double v[NVRED]) {
  const df kap(a.kappa);
  int kk[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    kk[c] = 3 * half + c;
    kk[3 + c] = 3 * (2 + half) + c;
  }
  // gamma5 (in - kappa hop): the second triple is a lower spin (sign -1)
  cpx<df> o[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const cpx<df> c = ldg_cdf(a.in, fin, s, kk[q]);
    cpx<df> t = c - kap * acc6[q];
    o[q] = q >= 3 ? -t : t;
    if (MODE == MODE_K) acc6[q] = c;   // keep the input for ||in||^2
  }
  const bool red = a.partials != nullptr;
  Acc<df> n0, n1;
  if constexpr (MODE == MODE_K) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      st_cdf(a.out, rhs, s, kk[q], o[q]);
      if (red) {
        acc_norm(n0, o[q]);
        acc_norm(n1, acc6[q]);
      }
    }
    v[0] = n0.get();
    v[1] = n1.get();
  } else if constexpr (MODE == MODE_R) {
    const df sg(a.sigma0), al(a.ms[rhs].alpha);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const cpx<df> p = ld_cdf(a.aux1, rhs, s, kk[q]);
      cpx<df> r = ld_cdf(a.aux2, rhs, s, kk[q]);
      r = r - al * (o[q] + sg * p);
      st_cdf(a.aux2, rhs, s, kk[q], r);
      if (red) acc_norm(n0, r);
    }
    v[0] = n0.get();
  } else if constexpr (MODE == MODE_LZK) {
    const df sc(a.lz[rhs].inv_n);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const cpx<df> t = sc * o[q];
      st_cdf(a.out, rhs, s, kk[q], t);
      if (red) acc_norm(n0, t);
    }
    v[0] = n0.get();
  } else if constexpr (MODE == MODE_LZL) {
    const LzRhs& L = a.lz[rhs];
    const int j = L.j;
    const df ca(L.a), cb(L.b);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      cpx<df> w = o[q] - ca * ld_cdf(a.aux1, j * a.nrhs + rhs, s, kk[q]);
      if (j > 0) w = w - cb * ld_cdf(a.aux1, (j - 1) * a.nrhs + rhs, s, kk[q]);
      st_cdf(a.out, (j + 1) * a.nrhs + rhs, s, kk[q], w);
      if (red) acc_norm(n0, w);
    }
    v[0] = n0.get();
  }
}

// 80 registers: no spills, 24 warps per SM (96: 20; 72 and 64 spill)
#ifndef OVL_WILSON_REG_PAIR
#define OVL_WILSON_REG_PAIR 80
#endif
template <int MODE>
__global__ void __maxnreg__(OVL_WILSON_REG_PAIR) wilson_pair_kernel(const DArgs a) {
  __shared__ double red[(256 / 32) * NVRED];
  const int half = threadIdx.x & 1;
  const int sb = blockIdx.x / a.ngr;
  const int rg = blockIdx.x - sb * a.ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + (threadIdx.x >> 1);
  bool live = s < a.g.V && rhs < a.nrhs;
  if (live && a.ms != nullptr && (MODE == MODE_K || MODE == MODE_R)) live = !a.ms[rhs].done;
  int fin = rhs;
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (live) live = !a.lz[rhs].done;
    if (MODE == MODE_LZK && live) fin = a.lz[rhs].j * a.nrhs + rhs;
  }
  double v[NVRED] = {0.0, 0.0, 0.0, 0.0};
  cpx<df> up[3], la[3], lb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) up[c] = la[c] = lb[c] = cmk(df(0.f), df(0.f));
  if (live) {
    int x[4];
    site_coords(a.g, s, x);
#pragma unroll 1
    for (int n = 0; n < 8; ++n) {
      const int mu = n >> 1;
      const bool fwd = (n & 1) == 0;
      const int sS = fwd ? 2 : 0;
      const bool lo3 = mu <= 1;
      // powers of i of the projection and of the lower-spin expansion (see hop_nb_df_core)
      const int a0 = (sS + (mu == 0 || mu == 2 ? 1 : mu == 1 ? 2 : 0)) & 3;
      const int a1 = (sS + (mu == 0 ? 1 : mu == 2 ? 3 : 0)) & 3;
      const int b0 = (sS + (mu == 0 || mu == 2 ? 3 : 0)) & 3;
      const int b1 = (sS + (mu == 0 ? 3 : mu == 1 ? 2 : mu == 2 ? 1 : 0)) & 3;
      const int other = half == 0 ? (lo3 ? 3 : 2) : (lo3 ? 2 : 3);
      const int ah = half == 0 ? a0 : a1;
      const int bh = half == 0 ? (lo3 ? b1 : b0) : (lo3 ? b0 : b1);
      const int sn = nb_site(a.g, x, s, n);
      cpx<df> h[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        h[c] = padd(ldg_cdf(a.in, fin, sn, 3 * half + c), ipow(ldg_cdf(a.in, fin, sn, 3 * other + c), ah));
      const float4* lp = reinterpret_cast<const float4*>(a.links.data) + (size_t)n * 9 * a.links.V + s;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        cpx<df> u[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float4 q = __ldg(lp + (size_t)(3 * r + b) * a.links.V);
          u[b] = cmk(df(q.x, q.y), df(q.z, q.w));
        }
        Dot2 re = dot2_first(u[0].r, h[0].r), im = dot2_first(u[0].r, h[0].i);
        dot2_add(re, -u[0].i, h[0].i);
        dot2_add(im, u[0].i, h[0].r);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
          dot2_add(re, u[b].r, h[b].r);
          dot2_add(re, -u[b].i, h[b].i);
          dot2_add(im, u[b].r, h[b].i);
          dot2_add(im, u[b].i, h[b].r);
        }
        const cpx<df> w = cmk(df(re.s, re.c), df(im.s, im.c));
        up[r] = padd(up[r], w);
        const cpx<df> wl = ipow(w, bh);
        if (lo3) la[r] = padd(la[r], wl);
        else lb[r] = padd(lb[r], wl);
      }
    }
  }
  // every lane of the warp takes part in the exchange (a pair shares s and rhs, so both of
  // its lanes are live or neither is)
  cpx<df> acc6[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc6[c] = up[c];
    acc6[3 + c] = lb[c] + shfl_pair(la[c]);
  }
  if (live) pair_epilogue<MODE>(a, rhs, fin, s, half, acc6, v);
  if (a.partials != nullptr) {
    double tot[NVRED];
    block_reduce_partials<double>(v, red, tot);
    if (threadIdx.x == 0 && rhs < a.nrhs) {
#pragma unroll
      for (int j = 0; j < NVRED; ++j) a.partials[((size_t)rhs * a.nsb + sb) * NVRED + j] = tot[j];
    }
  }
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (a.lzc.ctr != nullptr) lz_arrive<MODE>(a, rhs, a.nsb);
  }
}

// true when the lattice can be covered by whole variant-2 tiles
bool wilson_tiles_fit(const Geom& g) {
  return g.L[0] % TX == 0 && g.L[1] % TY == 0 && g.L[2] % TZ == 0 && g.L[3] % TT == 0;
}

// Variant 1 (direction split): a block of 4 * BX threads covers BX sites of one system;
// warp w handles direction w % 4 (forward and backward hop) for the 32 sites of group
// w / 4, so every thread walks two neighbours instead of eight and the direction is
// uniform within a warp. The four partial sums meet in shared memory and the
// direction-0 warps finish the site.
template <int MODE, int PIN, int PL, int POUT, int PA1, int PA2>
__global__ void __launch_bounds__(4 * BX) __maxnreg__((MaxReg<PL, PIN>::v)) wilson_split_kernel(const DArgs a) {
  using T = typename Real<PL>::T;
  __shared__ cpx<T> part[3][BX][12];
  __shared__ double red[(4 * BX / 32) * NVRED];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dir = warp & 3, grp = warp >> 2;
  const int sb = blockIdx.x / a.nrhs;
  const int rhs = blockIdx.x - sb * a.nrhs;
  const int sl = grp * 32 + lane;
  const int s = sb * BX + sl;
  bool live = s < a.g.V;
  if (live && a.ms != nullptr && (MODE == MODE_K || MODE == MODE_R)) live = !a.ms[rhs].done;
  int fin = rhs;
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (live) live = !a.lz[rhs].done;
    if (MODE == MODE_LZK && live) fin = a.lz[rhs].j * a.nrhs + rhs;
  }
  cpx<T> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cmk(T(0), T(0));
  if (live) {
    int x[4];
    site_coords(a.g, s, x);
    const int sy = a.g.L[0], sz = sy * a.g.L[1], st = sz * a.g.L[2];
    if (dir == 0) hop_dir<0, PIN, PL, T>(a.g, a.links, a.in, fin, s, x, 1, acc);
    else if (dir == 1) hop_dir<1, PIN, PL, T>(a.g, a.links, a.in, fin, s, x, sy, acc);
    else if (dir == 2) hop_dir<2, PIN, PL, T>(a.g, a.links, a.in, fin, s, x, sz, acc);
    else hop_dir<3, PIN, PL, T>(a.g, a.links, a.in, fin, s, x, st, acc);
  }
  if (dir != 0) {
#pragma unroll
    for (int k = 0; k < 12; ++k) part[dir - 1][sl][k] = acc[k];
  }
  __syncthreads();
  using R = typename RedT<T>::type;
  R v[NVRED] = {R(0), R(0), R(0), R(0)};
  if (dir == 0 && live) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = acc[k] + part[0][sl][k] + part[1][sl][k] + part[2][sl][k];
    wilson_epilogue<MODE, PIN, POUT, PA1, PA2, T>(a, rhs, fin, s, acc, v);
  }
  if (a.partials != nullptr) {
    double tot[NVRED];
    block_reduce_partials<R>(v, red, tot);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int j = 0; j < NVRED; ++j) a.partials[((size_t)rhs * a.nsb + sb) * NVRED + j] = tot[j];
    }
  }
  if constexpr (MODE == MODE_LZK || MODE == MODE_LZL) {
    if (a.lzc.ctr != nullptr) lz_arrive<MODE>(a, rhs, a.nsb);
  }
}

Shape make_shape(int V, int nrhs) {
  Shape s;
  s.nsb = (V + BX - 1) / BX;
  s.by = nrhs < 4 ? nrhs : 4;
  s.ngr = (nrhs + s.by - 1) / s.by;
  return s;
}

template <int MODE, int PIN, int PL, int POUT, int PA1, int PA2>
static void run(DArgs a, cudaStream_t st) {
  Shape sh = make_shape(a.g.V, a.nrhs);
  a.nsb = sh.nsb;
  a.ngr = sh.ngr;
  if constexpr (PIN == P64E && PL == P64E && POUT == P64E && PA1 == P64E && PA2 == P64E && MODE != MODE_OVL) {
    if (a.variant == 3) {
      // lane pairs over BX sites x up to 2 systems per block; partials keep the layout
      const int by = a.nrhs < 2 ? a.nrhs : 2;
      a.ngr = (a.nrhs + by - 1) / by;
      wilson_pair_kernel<MODE><<<dim3((unsigned)(sh.nsb * a.ngr)), dim3(2 * BX, by), 0, st>>>(a);
      return;
    }
  }
  if (a.variant == 1) {
    // one system per block; partials keep the (system, BX-site block) layout of variant 0
    wilson_split_kernel<MODE, PIN, PL, POUT, PA1, PA2><<<dim3((unsigned)(sh.nsb * a.nrhs)), dim3(4 * BX), 0, st>>>(a);
  } else if (a.variant == 2 && wilson_tiles_fit(a.g)) {
    const unsigned ntiles = (unsigned)(a.g.V / (TX * TY * TZ * TT));
    wilson_kernel<MODE, PIN, PL, POUT, PA1, PA2, true><<<dim3(ntiles, (unsigned)a.nrhs), dim3(TX * TY * TZ * TT), 0, st>>>(a);
  } else {
    wilson_kernel<MODE, PIN, PL, POUT, PA1, PA2, false><<<sh.grid(), sh.block(), 0, st>>>(a);
  }
}

static DArgs base_args(const Geom& g, double kappa, LinkRef links, int nrhs) {
  DArgs a;
  a.g = g;
  a.kappa = kappa;
  a.links = links;
  a.in = a.out = a.aux1 = a.aux2 = SpinorRef{nullptr, nullptr, g.V};
  a.nrhs = nrhs;
  a.nsb = a.ngr = 0;
  a.partials = nullptr;
  a.ms = nullptr;
  a.sigma0 = 0;
  a.c1 = a.c2 = 0;
  a.coef = nullptr;
  a.herm = 0;
  a.variant = nrhs >= 4 ? links.variant_multi : links.variant;
  a.lz = nullptr;
  a.lzc = LzCtl{nullptr, nullptr, nullptr, nullptr, 0, nullptr};
  return a;
}

#define OVL_BAD_COMBO() note_bad_combo(__func__)

void launch_wilson_K(int pin, int plink, int pout, const Geom& g, double kappa, LinkRef links, SpinorRef in,
                     SpinorRef out, int nrhs, double* partials, const MsRhs* ms, cudaStream_t st) {
  DArgs a = base_args(g, kappa, links, nrhs);
  a.in = in;
  a.out = out;
  a.partials = partials;
  a.ms = ms;
  if (pin == P64 && plink == P64 && pout == P64) run<MODE_K, P64, P64, P64, P64, P64>(a, st);
  else if (pin == P32 && plink == P32 && pout == P32) run<MODE_K, P32, P32, P32, P32, P32>(a, st);
  else if (pin == P16 && plink == P16 && pout == P16) run<MODE_K, P16, P16, P16, P16, P16>(a, st);
  else if (pin == P32 && plink == P16 && pout == P32) run<MODE_K, P32, P16, P32, P32, P32>(a, st);
  else if (pin == P32 && plink == P16 && pout == P16) run<MODE_K, P32, P16, P16, P32, P32>(a, st);
  else if (pin == P64E && plink == P64E && pout == P64E) run<MODE_K, P64E, P64E, P64E, P64E, P64E>(a, st);
  else OVL_BAD_COMBO();
}

void launch_wilson_mscg_r(int pt, int plink, int pr, int pp, const Geom& g, double kappa, LinkRef links,
                          SpinorRef t, SpinorRef p0, SpinorRef r, int nrhs, double sigma0, double* partials,
                          const MsRhs* ms, cudaStream_t st) {
  DArgs a = base_args(g, kappa, links, nrhs);
  a.in = t;
  a.aux1 = p0;
  a.aux2 = r;
  a.sigma0 = sigma0;
  a.partials = partials;
  a.ms = ms;
  if (pt == P64 && plink == P64 && pr == P64 && pp == P64) run<MODE_R, P64, P64, P64, P64, P64>(a, st);
  else if (pt == P32 && plink == P32 && pr == P32 && pp == P32) run<MODE_R, P32, P32, P32, P32, P32>(a, st);
  else if (pt == P16 && plink == P16 && pr == P32 && pp == P16) run<MODE_R, P16, P16, P32, P16, P32>(a, st);
  else if (pt == P64E && plink == P64E && pr == P64E && pp == P64E) run<MODE_R, P64E, P64E, P64E, P64E, P64E>(a, st);
  else OVL_BAD_COMBO();
}

void launch_wilson_lzK(int pw, int plink, int pt, const Geom& g, double kappa, LinkRef links, SpinorRef W,
                       SpinorRef t, int nrhs, double* partials, const LzCtl& ctl, cudaStream_t st) {
  DArgs a = base_args(g, kappa, links, nrhs);
  a.in = W;
  a.out = t;
  a.partials = partials;
  a.lz = ctl.lz;
  a.lzc = ctl;
  if (pw == P64 && plink == P64 && pt == P64) run<MODE_LZK, P64, P64, P64, P64, P64>(a, st);
  else if (pw == P32 && plink == P32 && pt == P32) run<MODE_LZK, P32, P32, P32, P32, P32>(a, st);
  else if (pw == P16 && plink == P16 && pt == P16) run<MODE_LZK, P16, P16, P16, P16, P16>(a, st);
  else if (pw == P64E && plink == P64E && pt == P64E) run<MODE_LZK, P64E, P64E, P64E, P64E, P64E>(a, st);
  else OVL_BAD_COMBO();
}

void launch_wilson_lzL(int pt, int plink, int pw, const Geom& g, double kappa, LinkRef links, SpinorRef t,
                       SpinorRef W, int nrhs, double* partials, const LzCtl& ctl, cudaStream_t st) {
  DArgs a = base_args(g, kappa, links, nrhs);
  a.in = t;
  a.out = W;
  a.aux1 = W;
  a.partials = partials;
  a.lz = ctl.lz;
  a.lzc = ctl;
  if (pt == P64 && plink == P64 && pw == P64) run<MODE_LZL, P64, P64, P64, P64, P64>(a, st);
  else if (pt == P32 && plink == P32 && pw == P32) run<MODE_LZL, P32, P32, P32, P32, P32>(a, st);
  else if (pt == P16 && plink == P16 && pw == P16) run<MODE_LZL, P16, P16, P16, P16, P16>(a, st);
  else if (pt == P64E && plink == P64E && pw == P64E) run<MODE_LZL, P64E, P64E, P64E, P64E, P64E>(a, st);
  else OVL_BAD_COMBO();
}

void launch_wilson_ovl(int py, int plink, int pv, const Geom& g, double kappa, LinkRef links, SpinorRef y,
                       SpinorRef v, SpinorRef out, SpinorRef w, int nrhs, double c1, double c2,
                       const double* coef, int herm, double* partials, cudaStream_t st) {
  DArgs a = base_args(g, kappa, links, nrhs);
  a.in = y;
  a.aux1 = v;
  a.out = out;
  a.aux2 = w;
  a.c1 = c1;
  a.c2 = c2;
  a.coef = coef;
  a.herm = herm;
  a.partials = partials;
  if (py == P64 && plink == P64 && pv == P64) run<MODE_OVL, P64, P64, P64, P64, P64>(a, st);
  else if (py == P32 && plink == P32 && pv == P32) run<MODE_OVL, P32, P32, P32, P32, P32>(a, st);
  else if (py == P32 && plink == P32 && pv == P64) run<MODE_OVL, P32, P32, P64, P64, P64>(a, st);
  else if (py == P32 && plink == P16 && pv == P32) run<MODE_OVL, P32, P16, P32, P32, P32>(a, st);
  else if (py == P32 && plink == P16 && pv == P64) run<MODE_OVL, P32, P16, P64, P64, P64>(a, st);
  else if (py == P64 && plink == P64 && pv == P32) run<MODE_OVL, P64, P64, P32, P32, P32>(a, st);
  else if (py == P64E && plink == P64E && pv == P64) run<MODE_OVL, P64E, P64E, P64, P64, P64>(a, st);
  else if (py == P64E && plink == P64E && pv == P32) run<MODE_OVL, P64E, P64E, P32, P32, P32>(a, st);
  else OVL_BAD_COMBO();
}

}  // namespace ovl
