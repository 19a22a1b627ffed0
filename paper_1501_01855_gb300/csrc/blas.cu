// Vector kernels of liboverlap: layout conversion, axpby, inner products,
// the fused SUMR step, and the block Gram / combination kernels of the Ritz step
// and the deflation projections. Every reduction writes per-(system, block)
// partials that are summed in a fixed order, so results do not depend on timing.
#include <stdio.h>

#include "kernels.h"

namespace ovl {

#define SITE_RHS_INDEX()                                   \
  const int sb = blockIdx.x / ngr;                         \
  const int rg = blockIdx.x - sb * ngr;                    \
  const int rhs = rg * blockDim.y + threadIdx.y;           \
  const int s = sb * BX + threadIdx.x;

// ---------------------------------------------------------------- pack / unpack
template <typename CT, int P>
__global__ void pack_kernel(const CT* canon, SpinorRef out, int nrhs, int V, int ngr) {
  SITE_RHS_INDEX();
  if (s >= V || rhs >= nrhs) return;
  const CT* c = canon + ((size_t)rhs * V + s) * 24;
  cpx<double> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = cmk((double)c[2 * k], (double)c[2 * k + 1]);
  store_spinor_any<P>(out, rhs, s, v);
}
template <typename CT, int P>
__global__ void unpack_kernel(CT* canon, SpinorRef in, int nrhs, int V, int ngr) {
  SITE_RHS_INDEX();
  if (s >= V || rhs >= nrhs) return;
  CT* c = canon + ((size_t)rhs * V + s) * 24;
  cpx<double> v[12];
  load_spinor_any<P>(in, rhs, s, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    c[2 * k] = (CT)v[k].r;
    c[2 * k + 1] = (CT)v[k].i;
  }
}

template <typename CT>
static void pack_t(const CT* canon, int p, SpinorRef out, int nrhs, int V, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (p == P64) pack_kernel<CT, P64><<<sh.grid(), sh.block(), 0, st>>>(canon, out, nrhs, V, sh.ngr);
  else if (p == P64E) pack_kernel<CT, P64E><<<sh.grid(), sh.block(), 0, st>>>(canon, out, nrhs, V, sh.ngr);
  else if (p == P32) pack_kernel<CT, P32><<<sh.grid(), sh.block(), 0, st>>>(canon, out, nrhs, V, sh.ngr);
  else pack_kernel<CT, P16><<<sh.grid(), sh.block(), 0, st>>>(canon, out, nrhs, V, sh.ngr);
}
template <typename CT>
static void unpack_t(CT* canon, int p, SpinorRef in, int nrhs, int V, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (p == P64) unpack_kernel<CT, P64><<<sh.grid(), sh.block(), 0, st>>>(canon, in, nrhs, V, sh.ngr);
  else if (p == P64E) unpack_kernel<CT, P64E><<<sh.grid(), sh.block(), 0, st>>>(canon, in, nrhs, V, sh.ngr);
  else if (p == P32) unpack_kernel<CT, P32><<<sh.grid(), sh.block(), 0, st>>>(canon, in, nrhs, V, sh.ngr);
  else unpack_kernel<CT, P16><<<sh.grid(), sh.block(), 0, st>>>(canon, in, nrhs, V, sh.ngr);
}

void launch_pack(int dtype, const void* canon, int pout, SpinorRef out, int nrhs, int V, cudaStream_t st) {
  if (dtype == 0) pack_t((const double*)canon, pout, out, nrhs, V, st);
  else pack_t((const float*)canon, pout, out, nrhs, V, st);
}
void launch_unpack(int dtype, void* canon, int pin, SpinorRef in, int nrhs, int V, cudaStream_t st) {
  if (dtype == 0) unpack_t((double*)canon, pin, in, nrhs, V, st);
  else unpack_t((float*)canon, pin, in, nrhs, V, st);
}

// ---------------------------------------------------------------- convert
template <int PI, int PO>
__global__ void convert_kernel(SpinorRef in, SpinorRef out, int nrhs, int V, int ngr) {
  SITE_RHS_INDEX();
  if (s >= V || rhs >= nrhs) return;
  cpx<double> v[12];
  load_spinor_any<PI>(in, rhs, s, v);
  store_spinor_any<PO>(out, rhs, s, v);
}
void launch_convert(int pin, SpinorRef in, int pout, SpinorRef out, int nrhs, int V, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
#define CONV(A, B) convert_kernel<A, B><<<sh.grid(), sh.block(), 0, st>>>(in, out, nrhs, V, sh.ngr)
  if (pin == P64 && pout == P32) CONV(P64, P32);
  else if (pin == P32 && pout == P64) CONV(P32, P64);
  else if (pin == P64 && pout == P64) CONV(P64, P64);
  else if (pin == P32 && pout == P32) CONV(P32, P32);
  else if (pin == P64 && pout == P16) CONV(P64, P16);
  else if (pin == P32 && pout == P16) CONV(P32, P16);
  else if (pin == P16 && pout == P32) CONV(P16, P32);
  else if (pin == P16 && pout == P64) CONV(P16, P64);
  else if (pin == P64 && pout == P64E) CONV(P64, P64E);
  else if (pin == P64E && pout == P64) CONV(P64E, P64);
  else if (pin == P32 && pout == P64E) CONV(P32, P64E);
  else if (pin == P64E && pout == P32) CONV(P64E, P32);
  else if (pin == P64E && pout == P64E) CONV(P64E, P64E);
  else CONV(P16, P16);
#undef CONV
}

// ---------------------------------------------------------------- axpby
template <int P>
__global__ void axpby_kernel(const double* a, const double* b, SpinorRef x, SpinorRef y, SpinorRef z, int nrhs,
                             int V, int ngr) {
  using T = typename Real<P>::T;
  SITE_RHS_INDEX();
  if (s >= V || rhs >= nrhs) return;
  const cpx<T> ca = cmk((T)a[2 * rhs], (T)a[2 * rhs + 1]);
  const cpx<T> cb = cmk((T)b[2 * rhs], (T)b[2 * rhs + 1]);
  cpx<T> xv[12], yv[12];
  load_spinor_as<P, T>(x, rhs, s, xv);
  load_spinor_as<P, T>(y, rhs, s, yv);
#pragma unroll
  for (int k = 0; k < 12; ++k) xv[k] = ca * xv[k] + cb * yv[k];
  store_spinor_as<P, T>(z, rhs, s, xv);
}
void launch_axpby(int p, const double* a, const double* b, SpinorRef x, SpinorRef y, SpinorRef z, int nrhs, int V,
                  cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (p == P64) axpby_kernel<P64><<<sh.grid(), sh.block(), 0, st>>>(a, b, x, y, z, nrhs, V, sh.ngr);
  else if (p == P32) axpby_kernel<P32><<<sh.grid(), sh.block(), 0, st>>>(a, b, x, y, z, nrhs, V, sh.ngr);
  else if (p == P64E) axpby_kernel<P64E><<<sh.grid(), sh.block(), 0, st>>>(a, b, x, y, z, nrhs, V, sh.ngr);
  else axpby_kernel<P16><<<sh.grid(), sh.block(), 0, st>>>(a, b, x, y, z, nrhs, V, sh.ngr);
}

// ---------------------------------------------------------------- dot / norm
template <int PX, int PY, bool NORM>
__global__ void __launch_bounds__(256) dot_kernel(SpinorRef x, SpinorRef y, int nrhs, int V, int nsb, int ngr,
                                                  double* partials) {
  __shared__ double red[4 * (BX / 32) * 2];
  SITE_RHS_INDEX();
  double v[2] = {0.0, 0.0};
  if (s < V && rhs < nrhs) {
    cpx<double> a[12];
    load_spinor_any<PX>(x, rhs, s, a);
    if (NORM) {
#pragma unroll
      for (int k = 0; k < 12; ++k) v[0] += norm2(a[k]);
    } else {
      cpx<double> b[12];
      load_spinor_any<PY>(y, rhs, s, b);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cpx<double> d = cmulc(a[k], b[k]);
        v[0] += d.r;
        v[1] += d.i;
      }
    }
  }
  block_reduce_rows<2>(v, red);
  if (threadIdx.x == 0 && rhs < nrhs) {
    partials[((size_t)rhs * nsb + sb) * NVRED + 0] = v[0];
    partials[((size_t)rhs * nsb + sb) * NVRED + 1] = v[1];
  }
}
void launch_dot(int px, SpinorRef x, int py, SpinorRef y, int nrhs, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
#define DOT(A, B) dot_kernel<A, B, false><<<sh.grid(), sh.block(), 0, st>>>(x, y, nrhs, V, sh.nsb, sh.ngr, partials)
  if (px == P64 && py == P64) DOT(P64, P64);
  else if (px == P32 && py == P32) DOT(P32, P32);
  else if (px == P64 && py == P32) DOT(P64, P32);
  else if (px == P32 && py == P64) DOT(P32, P64);
  else if (px == P64E && py == P64E) DOT(P64E, P64E);
  else if (px == P64 && py == P64E) DOT(P64, P64E);
  else if (px == P64E && py == P64) DOT(P64E, P64);
  else DOT(P16, P16);
#undef DOT
}
void launch_norm2(int px, SpinorRef x, int nrhs, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (px == P64) dot_kernel<P64, P64, true><<<sh.grid(), sh.block(), 0, st>>>(x, x, nrhs, V, sh.nsb, sh.ngr, partials);
  else if (px == P32) dot_kernel<P32, P32, true><<<sh.grid(), sh.block(), 0, st>>>(x, x, nrhs, V, sh.nsb, sh.ngr, partials);
  else if (px == P64E) dot_kernel<P64E, P64E, true><<<sh.grid(), sh.block(), 0, st>>>(x, x, nrhs, V, sh.nsb, sh.ngr, partials);
  else dot_kernel<P16, P16, true><<<sh.grid(), sh.block(), 0, st>>>(x, x, nrhs, V, sh.nsb, sh.ngr, partials);
}

__global__ void reduce_partials_kernel(const double* partials, int nsb, double* out) {
  __shared__ double sh[NVRED][128];
  const int rhs = blockIdx.x;
  // four site blocks in flight per thread, their sums combined in a fixed order
  double a4[4][NVRED];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int j = 0; j < NVRED; ++j) a4[u][j] = 0.0;
  int b = threadIdx.x;
  for (; b + 3 * (int)blockDim.x < nsb; b += 4 * blockDim.x) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < NVRED; ++j) a4[u][j] += partials[((size_t)rhs * nsb + b + u * blockDim.x) * NVRED + j];
  }
  for (int u = 0; b < nsb; b += blockDim.x, ++u)
#pragma unroll
    for (int j = 0; j < NVRED; ++j) a4[u & 3][j] += partials[((size_t)rhs * nsb + b) * NVRED + j];
  double a[NVRED];
#pragma unroll
  for (int j = 0; j < NVRED; ++j) a[j] = (a4[0][j] + a4[1][j]) + (a4[2][j] + a4[3][j]);
#pragma unroll
  for (int j = 0; j < NVRED; ++j) sh[j][threadIdx.x] = a[j];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int j = 0; j < NVRED; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NVRED; ++j) out[NVRED * rhs + j] = sh[j][0];
  }
}
void launch_reduce_partials(const double* partials, int nsb, int nrhs, double* out, cudaStream_t st) {
  reduce_partials_kernel<<<nrhs, 128, 0, st>>>(partials, nsb, out);
}

// ---------------------------------------------------------------- gamma5 / zero
template <int P>
__global__ void gamma5_kernel(SpinorRef x, int nrhs, int V, int ngr) {
  using T = typename Real<P>::T;
  SITE_RHS_INDEX();
  if (s >= V || rhs >= nrhs) return;
  cpx<T> v[12];
  load_spinor_as<P, T>(x, rhs, s, v);
#pragma unroll
  for (int k = 6; k < 12; ++k) v[k] = -v[k];
  store_spinor_as<P, T>(x, rhs, s, v);
}
void launch_gamma5(int p, SpinorRef x, int nrhs, int V, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (p == P64) gamma5_kernel<P64><<<sh.grid(), sh.block(), 0, st>>>(x, nrhs, V, sh.ngr);
  else if (p == P32) gamma5_kernel<P32><<<sh.grid(), sh.block(), 0, st>>>(x, nrhs, V, sh.ngr);
  else if (p == P64E) gamma5_kernel<P64E><<<sh.grid(), sh.block(), 0, st>>>(x, nrhs, V, sh.ngr);
  else gamma5_kernel<P16><<<sh.grid(), sh.block(), 0, st>>>(x, nrhs, V, sh.ngr);
}
void launch_zero(int p, SpinorRef x, int nrhs, int V, cudaStream_t st) {
  const size_t per = (size_t)V * spinor_site_bytes(p);
  cudaMemsetAsync(x.data, 0, per * nrhs, st);
  if (p == P16 && x.norm) cudaMemsetAsync(x.norm, 0, sizeof(float) * V * nrhs, st);
}

// ---------------------------------------------------------------- SUMR step
template <int P>
__global__ void __launch_bounds__(256) sumr_update_kernel(const double* sc, const int* active, SpinorRef x,
                                                          SpinorRef q, SpinorRef qt, SpinorRef pv, SpinorRef S,
                                                          SpinorRef u, int nrhs, int V, int nsb, int ngr,
                                                          double* partials) {
  using T = typename Real<P>::T;
  __shared__ double red[4 * (BX / 32) * 2];
  SITE_RHS_INDEX();
  double nq[2] = {0.0, 0.0};
  if (s < V && rhs < nrhs && active[rhs]) {
    const double* c = sc + 18 * rhs;
    const cpx<T> Rm1 = cmk((T)c[0], (T)c[1]), gs = cmk((T)c[2], (T)c[3]), iR = cmk((T)c[4], (T)c[5]);
    const cpx<T> sgp = cmk((T)c[6], (T)c[7]), zm1 = cmk((T)c[8], (T)c[9]), gj = cmk((T)c[10], (T)c[11]);
    const cpx<T> gam = cmk((T)c[12], (T)c[13]), isg = cmk((T)c[14], (T)c[15]), sg = cmk((T)c[16], (T)c[17]);
    cpx<T> qv[12], qtv[12], pvv[12], Sv[12], uv[12], xv[12];
    load_spinor_as<P, T>(q, rhs, s, qv);
    load_spinor_as<P, T>(qt, rhs, s, qtv);
    load_spinor_as<P, T>(pv, rhs, s, pvv);
    load_spinor_as<P, T>(S, rhs, s, Sv);
    load_spinor_as<P, T>(u, rhs, s, uv);
    load_spinor_as<P, T>(x, rhs, s, xv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cpx<T> pn = (qv[k] - Rm1 * pvv[k] + gs * Sv[k]) * iR;
      Sv[k] = sgp * Sv[k] + zm1 * pvv[k];
      pvv[k] = pn;
      xv[k] = xv[k] + gj * pn;
      const cpx<T> qn = (uv[k] + gam * qtv[k]) * isg;
      qtv[k] = sg * qtv[k] + cmulc(gam, qn);
      qv[k] = qn;
      nq[0] += (double)norm2(qn);
    }
    store_spinor_as<P, T>(q, rhs, s, qv);
    store_spinor_as<P, T>(qt, rhs, s, qtv);
    store_spinor_as<P, T>(pv, rhs, s, pvv);
    store_spinor_as<P, T>(S, rhs, s, Sv);
    store_spinor_as<P, T>(x, rhs, s, xv);
  }
  if (partials != nullptr) {
    block_reduce_rows<2>(nq, red);
    if (threadIdx.x == 0 && rhs < nrhs) {
      partials[((size_t)rhs * nsb + sb) * NVRED + 0] = nq[0];
      partials[((size_t)rhs * nsb + sb) * NVRED + 1] = 0.0;
    }
  }
}
void launch_sumr_update(int p, const double* sc, const int* active, SpinorRef x, SpinorRef q, SpinorRef qt,
                        SpinorRef pv, SpinorRef S, SpinorRef u, int nrhs, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (p == P64)
    sumr_update_kernel<P64><<<sh.grid(), sh.block(), 0, st>>>(sc, active, x, q, qt, pv, S, u, nrhs, V, sh.nsb, sh.ngr, partials);
  else
    sumr_update_kernel<P32><<<sh.grid(), sh.block(), 0, st>>>(sc, active, x, q, qt, pv, S, u, nrhs, V, sh.nsb, sh.ngr, partials);
}

// ---------------------------------------------------------------- multi-mass SUMR step
// One Alg. 1 basis per source shared by nm masses (rho_k + V has the Krylov space of V):
// for every active system (k, j) = k ns + j the per-mass update of p, S and x with its own
// coefficients sc[18 (k ns + j) ...] (the layout of sumr_update), then the shared
// q, q~ update of source j with scq[6 j ...] = (gamma_j, 1/sigma_j, sigma_j). partials
// {||q||^2} per source.
template <int P>
__global__ void __launch_bounds__(256) sumr_mm_update_kernel(const double* sc, const double* scq, const int* active,
                                                             const int* qactive, SpinorRef x, SpinorRef q,
                                                             SpinorRef qt, SpinorRef pv, SpinorRef S, SpinorRef u,
                                                             int ns, int nm, int V, int nsb, int ngr,
                                                             double* partials) {
  using T = typename Real<P>::T;
  __shared__ double red[4 * (BX / 32) * 2];
  SITE_RHS_INDEX();
  const int j = rhs;
  double nq[2] = {0.0, 0.0};
  if (s < V && j < ns && qactive[j]) {
    cpx<T> qv[12], qtv[12], uv[12];
    load_spinor_as<P, T>(q, j, s, qv);
    for (int k = 0; k < nm; ++k) {
      const int sys = k * ns + j;
      if (!active[sys]) continue;
      const double* c = sc + 18 * sys;
      const cpx<T> Rm1 = cmk((T)c[0], (T)c[1]), gs = cmk((T)c[2], (T)c[3]), iR = cmk((T)c[4], (T)c[5]);
      const cpx<T> sgp = cmk((T)c[6], (T)c[7]), zm1 = cmk((T)c[8], (T)c[9]), gj = cmk((T)c[10], (T)c[11]);
      cpx<T> pvv[12], Sv[12], xv[12];
      load_spinor_as<P, T>(pv, sys, s, pvv);
      load_spinor_as<P, T>(S, sys, s, Sv);
      load_spinor_as<P, T>(x, sys, s, xv);
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        const cpx<T> pn = (qv[m] - Rm1 * pvv[m] + gs * Sv[m]) * iR;
        Sv[m] = sgp * Sv[m] + zm1 * pvv[m];
        pvv[m] = pn;
        xv[m] = xv[m] + gj * pn;
      }
      store_spinor_as<P, T>(pv, sys, s, pvv);
      store_spinor_as<P, T>(S, sys, s, Sv);
      store_spinor_as<P, T>(x, sys, s, xv);
    }
    load_spinor_as<P, T>(qt, j, s, qtv);
    load_spinor_as<P, T>(u, j, s, uv);
    const double* cq = scq + 6 * j;
    const cpx<T> gam = cmk((T)cq[0], (T)cq[1]), isg = cmk((T)cq[2], (T)cq[3]), sg = cmk((T)cq[4], (T)cq[5]);
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const cpx<T> qn = (uv[m] + gam * qtv[m]) * isg;
      qtv[m] = sg * qtv[m] + cmulc(gam, qn);
      qv[m] = qn;
      nq[0] += (double)norm2(qn);
    }
    store_spinor_as<P, T>(q, j, s, qv);
    store_spinor_as<P, T>(qt, j, s, qtv);
  }
  if (partials != nullptr) {
    block_reduce_rows<2>(nq, red);
    if (threadIdx.x == 0 && j < ns) {
      partials[((size_t)j * nsb + sb) * NVRED + 0] = nq[0];
      partials[((size_t)j * nsb + sb) * NVRED + 1] = 0.0;
    }
  }
}
void launch_sumr_mm_update(int p, const double* sc, const double* scq, const int* active, const int* qactive,
                           SpinorRef x, SpinorRef q, SpinorRef qt, SpinorRef pv, SpinorRef S, SpinorRef u, int ns,
                           int nm, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, ns);
  if (p == P64)
    sumr_mm_update_kernel<P64><<<sh.grid(), sh.block(), 0, st>>>(sc, scq, active, qactive, x, q, qt, pv, S, u, ns,
                                                                  nm, V, sh.nsb, sh.ngr, partials);
  else
    sumr_mm_update_kernel<P32><<<sh.grid(), sh.block(), 0, st>>>(sc, scq, active, qactive, x, q, qt, pv, S, u, ns,
                                                                  nm, V, sh.nsb, sh.ngr, partials);
}

// ---------------------------------------------------------------- Gram block
// G[i, j] = sum over sites of (A_i, g5? B_j). Grid: (tiles of 16 x 16 pairs) x
// (site ranges); each block stages SC sites of its 16 A and 16 B vectors in shared
// memory as FP32 and accumulates every pair in FP32 over one stage, then in FP64.
constexpr int GT = 16, GSC = 8;
template <int PA, int PB>
__global__ void __launch_bounds__(256) gram_kernel(SpinorRef A, int na, SpinorRef B, int nb, int V, int nrange,
                                                   int g5, double* work) {
  __shared__ cpx<float> sa[GT][GSC][12];
  __shared__ cpx<float> sbm[GT][GSC][12];
  const int ntj = (nb + GT - 1) / GT;
  const int tile = blockIdx.x;
  const int ti = tile / ntj, tj = tile - ti * ntj;
  const int range = blockIdx.y;
  const int s0 = (int)(((long long)V * range) / nrange);
  const int s1 = (int)(((long long)V * (range + 1)) / nrange);
  const int li = threadIdx.x / GT, lj = threadIdx.x % GT;
  const int gi = ti * GT + li, gj = tj * GT + lj;
  double accr = 0.0, acci = 0.0;
  for (int base = s0; base < s1; base += GSC) {
    // stage: 256 threads load GT*GSC site-vectors of A and of B
    for (int e = threadIdx.x; e < GT * GSC; e += blockDim.x) {
      const int vi = e / GSC, so = e % GSC;
      const int s = base + so;
      cpx<double> w[12];
      const int ia = ti * GT + vi, jb = tj * GT + vi;
      if (s < s1 && ia < na) {
        load_spinor_any<PA>(A, ia, s, w);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = cmk(0.0, 0.0);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) sa[vi][so][k] = cmk((float)w[k].r, (float)w[k].i);
      if (s < s1 && jb < nb) {
        load_spinor_any<PB>(B, jb, s, w);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = cmk(0.0, 0.0);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cpx<float> q = cmk((float)w[k].r, (float)w[k].i);
        if (g5 && k >= 6) q = -q;
        sbm[vi][so][k] = q;
      }
    }
    __syncthreads();
    float fr = 0.f, fi = 0.f;
#pragma unroll
    for (int so = 0; so < GSC; ++so) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cpx<float> a = sa[li][so][k], b = sbm[lj][so][k];
        fr += a.r * b.r + a.i * b.i;
        fi += a.r * b.i - a.i * b.r;
      }
    }
    accr += fr;
    acci += fi;
    __syncthreads();
  }
  if (gi < na && gj < nb) {
    work[(((size_t)range * na + gi) * nb + gj) * 2] = accr;
    work[(((size_t)range * na + gi) * nb + gj) * 2 + 1] = acci;
  }
}
__global__ void gram_reduce_kernel(const double* work, int nrange, int nn, double* G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  double r = 0.0, i = 0.0;
  for (int k = 0; k < nrange; ++k) {
    r += work[((size_t)k * nn + e) * 2];
    i += work[((size_t)k * nn + e) * 2 + 1];
  }
  G[2 * e] += r;
  G[2 * e + 1] += i;
}
void launch_gram(int pa, SpinorRef A, int na, int pb, SpinorRef B, int nb, int V, double* G, double* work,
                 size_t work_doubles, int g5, cudaStream_t st) {
  const int nti = (na + GT - 1) / GT, ntj = (nb + GT - 1) / GT;
  int nrange = (int)(work_doubles / ((size_t)na * nb * 2));
  const int want = (304 * 4 + nti * ntj - 1) / (nti * ntj);
  if (nrange > want) nrange = want;
  if (nrange > V / GSC) nrange = V / GSC;
  if (nrange < 1) nrange = 1;
  dim3 grid(nti * ntj, nrange);
#define GRAM(X, Y) gram_kernel<X, Y><<<grid, 256, 0, st>>>(A, na, B, nb, V, nrange, g5, work)
  if (pa == P64 && pb == P64) GRAM(P64, P64);
  else if (pa == P32 && pb == P32) GRAM(P32, P32);
  else if (pa == P64 && pb == P32) GRAM(P64, P32);
  else GRAM(P32, P64);
#undef GRAM
  const int nn = na * nb;
  gram_reduce_kernel<<<(nn + 255) / 256, 256, 0, st>>>(work, nrange, nn, G);
}

// ---------------------------------------------------------------- combine
template <int PA, int PY>
__global__ void __launch_bounds__(256) combine_kernel(SpinorRef A, int na, const double* C, SpinorRef Y, int ny,
                                                      int V, int ngr, int add) {
  using T = typename Real<PY>::T;
  SITE_RHS_INDEX();
  const int j = rhs;
  if (s >= V || j >= ny) return;
  cpx<T> acc[12], a[12];
  if (add) {
    load_spinor_as<PY, T>(Y, j, s, acc);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = cmk(T(0), T(0));
  }
  for (int i = 0; i < na; ++i) {
    load_spinor_as<PA, T>(A, i, s, a);
    const cpx<T> c = cmk((T)C[2 * ((size_t)i * ny + j)], (T)C[2 * ((size_t)i * ny + j) + 1]);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = acc[k] + c * a[k];
  }
  store_spinor_as<PY, T>(Y, j, s, acc);
}
void launch_combine(int pa, SpinorRef A, int na, const double* C, int py, SpinorRef Y, int ny, int V, int add,
                    cudaStream_t st) {
  Shape sh = make_shape(V, ny);
#define COMB(X, Z) combine_kernel<X, Z><<<sh.grid(), sh.block(), 0, st>>>(A, na, C, Y, ny, V, sh.ngr, add)
  if (pa == P64 && py == P64) COMB(P64, P64);
  else if (pa == P32 && py == P32) COMB(P32, P32);
  else if (pa == P32 && py == P64) COMB(P32, P64);
  else COMB(P64, P32);
#undef COMB
}

// ---------------------------------------------------------------- FP32 issue probe
// Eight independent FMA chains per thread (enough to cover the FMA latency at full
// occupancy), so that the measured rate is the FP32 pipes' instruction issue rate.
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float* out) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  const float b = 0.999f, cc = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], b, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
void launch_fma_probe(int nblocks, int iters, float* out, cudaStream_t st) {
  fma_probe_kernel<<<nblocks, 256, 0, st>>>(iters, out);
}

}  // namespace ovl
