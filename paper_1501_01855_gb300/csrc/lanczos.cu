// Stored-basis Lanczos evaluation of the Zolotarev sum (Sec. 3):
//
//   y = sum_i omega_i (K^2 + sigma_i)^-1 v,   eps(K) v = K y.
//
// Every shifted system has the same Krylov space K_k(K^2, v), and its Galerkin (CG)
// solution after k steps is x_i = ||v|| V_k (T_k + sigma_i)^-1 e_1, with V_k the Lanczos
// basis and T_k the tridiagonal matrix of the recurrence. The multi-shift CG of mscg.cu
// carries one search direction per pole and updates all of them every step (two spinor
// passes per active pole and step); here the basis itself is kept in HBM instead, one
// vector per step, so that a step is two Wilson launches (their last blocks do the
// scalar work), and y comes at the end from N_Z tridiagonal solves (scalars) and a single
// pass over the stored vectors.
//
// Per step j (lz[rhs].j = j, unnormalised vectors W_l with v_l = W_l / n_l), two Wilson
// launches whose last block per system also runs the scalar step (dslash.cu, lz_finish):
//   MODE_LZK   t = K v_j;  alpha_j = ||t||^2,  a = alpha_j / n_j,  b = beta_{j-1} / n_{j-1}
//   MODE_LZL   W_{j+1} = K t - a W_j - b W_{j-1};  beta_j = ||W_{j+1}|| = n_{j+1}, for every
//              pole the LDL^T pivot d_j = alpha_j + sigma_i - beta_{j-1}^2 / d_{j-1} and the
//              residual norm rho_i <- rho_i beta_j / d_j of its Galerkin solution
//              (||r_i|| = ||v|| prod_l beta_l / d_l), the error bound sum_i |w_i| g_i rho_i
//              and the stopping test.
// The stopping rule is the one of the multi-shift CG (pole i contributes at most
// |w_i| g_i ||r_i|| to the error of eps(K) v, g_i = max_[a,b] x / (x^2 + sigma_i)); all
// poles keep improving until the sum is within eta ||v||.
//
// A cycle holds at most cap vectors. When it fills up, every pole's residual is
// r_i = -||v|| (T_k + sigma_i)^-1_{k-1,0} W_k, parallel to the last vector, so the rest
// of the sum is the same problem started from W_k with weights w_i ||v|| (-y_i,k-1): the
// cycle's part of y is added and the next cycle starts there.
#include "kernels.h"

namespace ovl {

// Fixed-order sum over the site-block partials (slot 0) of one system.
__device__ __forceinline__ double lz_sum_partials(const double* partials, int nsb, int rhs) {
  __shared__ double sh[128];
  double a = 0.0;
  for (int b = threadIdx.x; b < nsb; b += blockDim.x) a += partials[((size_t)rhs * nsb + b) * NVRED];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- init / restart
template <int PV, int PW, int PY>
__global__ void __launch_bounds__(256) lz_init_kernel(SpinorRef v, SpinorRef W, SpinorRef y, int nrhs, int V,
                                                      int nsb, int ngr, double* partials) {
  using T = typename Real<PW>::T;
  __shared__ double red[4 * (BX / 32) * 2];
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (s < V && rhs < nrhs) {
    cpx<T> a[12];
    load_spinor_as<PV, T>(v, rhs, s, a);
    store_spinor_as<PW, T>(W, rhs, s, a);
    // the norm of the stored (rounded) start vector, which the recurrence sees
    load_spinor_as<PW, T>(W, rhs, s, a);
    cpx<double> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[0] += to_d(a[k].r) * to_d(a[k].r) + to_d(a[k].i) * to_d(a[k].i);
      z[k] = cmk(0.0, 0.0);
    }
    store_spinor_any<PY>(y, rhs, s, z);
  }
  block_reduce_rows<2>(acc, red);
  if (threadIdx.x == 0 && rhs < nrhs) {
    partials[((size_t)rhs * nsb + sb) * NVRED + 0] = acc[0];
    partials[((size_t)rhs * nsb + sb) * NVRED + 1] = 0.0;
  }
}

void launch_lz_init(int pv, int pw, int py, SpinorRef v, SpinorRef W, SpinorRef y, int nrhs, int V,
                    double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
#define LZI(A, B, C) lz_init_kernel<A, B, C><<<sh.grid(), sh.block(), 0, st>>>(v, W, y, nrhs, V, sh.nsb, sh.ngr, partials)
  if (pv == P64 && pw == P64 && py == P64) LZI(P64, P64, P64);
  else if (pv == P64 && pw == P64E && py == P64E) LZI(P64, P64E, P64E);
  else if (pv == P32 && pw == P64E && py == P64E) LZI(P32, P64E, P64E);
  else if (pv == P64 && pw == P32 && py == P32) LZI(P64, P32, P32);
  else if (pv == P32 && pw == P32 && py == P32) LZI(P32, P32, P32);
  else if (pv == P64 && pw == P16 && py == P32) LZI(P64, P16, P32);
  else if (pv == P32 && pw == P16 && py == P32) LZI(P32, P16, P32);
  else if (pv == P32 && pw == P64 && py == P64) LZI(P32, P64, P64);
  else note_bad_combo("lz_init");
#undef LZI
}

// W_0 = W_j for the systems whose cycle filled up (status 3); partials of ||W_0||^2.
template <int PW>
__global__ void __launch_bounds__(256) lz_restart_kernel(SpinorRef W, const LzRhs* lz, int nrhs, int V, int nsb,
                                                         int ngr, double* partials) {
  using T = typename Real<PW>::T;
  __shared__ double red[4 * (BX / 32) * 2];
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (s < V && rhs < nrhs && !lz[rhs].finished && lz[rhs].status == 3) {
    cpx<T> a[12];
    load_spinor_as<PW, T>(W, lz[rhs].j * nrhs + rhs, s, a);
    store_spinor_as<PW, T>(W, rhs, s, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0] += to_d(a[k].r) * to_d(a[k].r) + to_d(a[k].i) * to_d(a[k].i);
  }
  block_reduce_rows<2>(acc, red);
  if (threadIdx.x == 0 && rhs < nrhs) {
    partials[((size_t)rhs * nsb + sb) * NVRED + 0] = acc[0];
    partials[((size_t)rhs * nsb + sb) * NVRED + 1] = 0.0;
  }
}

void launch_lz_restart(int pw, SpinorRef W, const LzRhs* lz, int nrhs, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (pw == P64) lz_restart_kernel<P64><<<sh.grid(), sh.block(), 0, st>>>(W, lz, nrhs, V, sh.nsb, sh.ngr, partials);
  else if (pw == P64E) lz_restart_kernel<P64E><<<sh.grid(), sh.block(), 0, st>>>(W, lz, nrhs, V, sh.nsb, sh.ngr, partials);
  else if (pw == P32) lz_restart_kernel<P32><<<sh.grid(), sh.block(), 0, st>>>(W, lz, nrhs, V, sh.nsb, sh.ngr, partials);
  else lz_restart_kernel<P16><<<sh.grid(), sh.block(), 0, st>>>(W, lz, nrhs, V, sh.nsb, sh.ngr, partials);
}

// ---------------------------------------------------------------- scalars
// Start a cycle: n_0 = ||W_0||. First cycle: weights omega_i and the budget eta ||v||
// (|eta|: the sign of eta selects the multi-shift CG's rule and does not matter here).
// Later cycles keep the weights set by lz_coef and the budget.
__global__ void lz_start_kernel(LzRhs* lz, const double* partials, int nsb, const Poles* P, const double* eta,
                                int maxit, int cap, int first) {
  const int rhs = blockIdx.x;
  LzRhs& L = lz[rhs];
  const double nn = lz_sum_partials(partials, nsb, rhs);
  if (!first && (L.finished || L.status != 3)) return;
  const double n0 = sqrt(nn);
  for (int i = threadIdx.x; i < P->n; i += blockDim.x) {
    if (first) L.w[i] = P->omega[i];
    L.d[i] = 0.0;
    L.rho[i] = n0;
  }
  if (threadIdx.x == 0) {
    if (first) {
      L.thr = fabs(eta[rhs]) * n0;
      L.even = eta[rhs] < 0.0 ? 1 : 0;
      L.total = 0;
      L.maxit = maxit;
      L.cycles = 0;
      L.finished = 0;
      L.w_reads = 0;
    }
    L.cap = cap;
    L.vnorm = n0;
    L.inv_n = n0 > 0.0 ? 1.0 / n0 : 0.0;
    L.inv_nprev = 0.0;
    L.a = L.b = L.alpha = L.beta_prev = 0.0;
    L.err = 0.0;
    L.j = 0;
    L.status = 0;
    L.cycles += 1;
    // nothing left to do: a zero vector (or, on a restart, a remainder already within budget)
    L.done = (n0 == 0.0) ? 1 : 0;
    if (L.done) L.finished = 1;
  }
}

void launch_lz_start(LzRhs* lz, const double* partials, int nsb, int nrhs, const Poles* poles, const double* eta,
                     int maxit, int cap, int first, cudaStream_t st) {
  lz_start_kernel<<<nrhs, 128, 0, st>>>(lz, partials, nsb, poles, eta, maxit, cap, first);
}
// ---------------------------------------------------------------- coefficients
// One block per system. Thread i (pole) solves (T_k + sigma_i) y_i = e_1 by the LDL^T
// factorisation of T_k + sigma_i (pivots d_l; L unit lower bidiagonal with l_l =
// beta_l / d_l): forward z_0 = 1, z_l = -(beta_{l-1} / d_{l-1}) z_{l-1}; back
// y_{k-1} = z_{k-1} / d_{k-1}, y_l = z_l / d_l - (beta_l / d_l) y_{l+1}. Y holds 2 cap
// doubles per pole and system (y, then the pivots). Then coefW_l = n_0 sum_i w_i y_il / n_l
// is the coefficient of the stored W_l in y. A cycle that filled up passes its remainder
// on: w_i <- w_i n_0 (-y_i,k-1).
__global__ void lz_coef_kernel(LzRhs* lz, const double* ahist, const double* bhist, int cap, const Poles* P,
                               double* Y, double* coefW) {
  const int rhs = blockIdx.x;
  LzRhs& L = lz[rhs];
  const int k = L.j;
  const int np = P->n;
  const double* al = ahist + (size_t)rhs * cap;
  const double* be = bhist + (size_t)rhs * cap;
  double* Yr = Y + (size_t)rhs * np * 2 * cap;
  double* cw = coefW + (size_t)rhs * cap;
  const bool active = k > 0 && L.status != 2;
  for (int i = threadIdx.x; i < np && active; i += blockDim.x) {
    const double sg = P->sigma0 + P->ds[i];
    double* y = Yr + (size_t)i * 2 * cap;
    double* d = y + cap;
    d[0] = al[0] + sg;
    double z = 1.0;
    y[0] = z / d[0];
    for (int l = 1; l < k; ++l) {
      d[l] = al[l] + sg - be[l - 1] * be[l - 1] / d[l - 1];
      z = -(be[l - 1] / d[l - 1]) * z;
      y[l] = z / d[l];
    }
    const double last = y[k - 1];
    for (int l = k - 2; l >= 0; --l) y[l] -= (be[l] / d[l]) * y[l + 1];
    const double wi = L.w[i];
    for (int l = 0; l < k; ++l) y[l] *= wi;
    if (L.status == 3) L.w[i] = wi * L.vnorm * (-last);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < cap; l += blockDim.x) {
    double c = 0.0;
    if (active && l < k) {
      for (int i = 0; i < np; ++i) c += Yr[(size_t)i * 2 * cap + l];
      const double nl = l == 0 ? L.vnorm : be[l - 1];
      c = nl > 0.0 ? L.vnorm * c / nl : 0.0;
    }
    cw[l] = c;
  }
}

void launch_lz_coef(LzRhs* lz, const double* ahist, const double* bhist, int cap, const Poles* poles, double* Y,
                    double* coefW, int nrhs, cudaStream_t st) {
  lz_coef_kernel<<<nrhs, 64, 0, st>>>(lz, ahist, bhist, cap, poles, Y, coefW);
}

// ---------------------------------------------------------------- combine
// y += sum_{l < k} coefW_l W_l. Double-float: chunk-major (one complex component of y at
// a time, every stored vector's chunk read once), coefficients converted to double-float
// once per block in shared memory.
__global__ void __launch_bounds__(256) lz_combine_df_kernel(SpinorRef W, SpinorRef y, const double* coefW,
                                                            const LzRhs* lz, int cap, int nrhs, int V, int ngr) {
  extern __shared__ float2 cf[];   // [blockDim.y][cap]
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const bool in_rhs = rhs < nrhs;
  const int k = in_rhs ? lz[rhs].j : 0;
  float2* c = cf + (size_t)threadIdx.y * cap;
  if (in_rhs) {
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
      const double v = coefW[(size_t)rhs * cap + l];
      const float h = (float)v;
      c[l] = make_float2(h, (float)(v - (double)h));
    }
  }
  __syncthreads();
  const int s = sb * BX + threadIdx.x;
  if (s >= V || !in_rhs || k == 0) return;
  const size_t Vs = (size_t)V;
  const float4* Wb = reinterpret_cast<const float4*>(W.data) + (size_t)rhs * 12 * Vs + s;
  float4* yy = reinterpret_cast<float4*>(y.data) + (size_t)rhs * 12 * Vs + s;
  const size_t slot = (size_t)nrhs * 12 * Vs;
  for (int q = 0; q < 12; ++q) {
    const float4 yw = yy[(size_t)q * Vs];
    cpx<df> acc = cmk(df(yw.x, yw.y), df(yw.z, yw.w));
    for (int l = 0; l < k; ++l) {
      const float4 w = __ldg(Wb + (size_t)l * slot + (size_t)q * Vs);
      const df cl(c[l].x, c[l].y);
      acc = acc + cmk(cl * df(w.x, w.y), cl * df(w.z, w.w));
    }
    yy[(size_t)q * Vs] = make_float4(acc.r.hi, acc.r.lo, acc.i.hi, acc.i.lo);
  }
}

// Other precisions: whole spinors, accumulated in the compute type of y.
template <int PW, int PY>
__global__ void __launch_bounds__(256) lz_combine_kernel(SpinorRef W, SpinorRef y, const double* coefW,
                                                         const LzRhs* lz, int cap, int nrhs, int V, int ngr) {
  using T = typename Real<PY>::T;
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  if (s >= V || rhs >= nrhs) return;
  const int k = lz[rhs].j;
  if (k == 0) return;
  cpx<T> acc[12], w[12];
  load_spinor_as<PY, T>(y, rhs, s, acc);
  for (int l = 0; l < k; ++l) {
    load_spinor_as<PW, T>(W, l * nrhs + rhs, s, w);
    const T cl = (T)coefW[(size_t)rhs * cap + l];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = acc[q] + cl * w[q];
  }
  store_spinor_as<PY, T>(y, rhs, s, acc);
}

void launch_lz_combine(int pw, int py, SpinorRef W, SpinorRef y, const double* coefW, const LzRhs* lz, int cap,
                       int nrhs, int V, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (pw == P64E && py == P64E) {
    const size_t smem = sizeof(float2) * (size_t)sh.by * cap;
    lz_combine_df_kernel<<<sh.grid(), sh.block(), smem, st>>>(W, y, coefW, lz, cap, nrhs, V, sh.ngr);
    return;
  }
#define LZC(A, B) lz_combine_kernel<A, B><<<sh.grid(), sh.block(), 0, st>>>(W, y, coefW, lz, cap, nrhs, V, sh.ngr)
  if (pw == P64 && py == P64) LZC(P64, P64);
  else if (pw == P32 && py == P32) LZC(P32, P32);
  else if (pw == P16 && py == P32) LZC(P16, P32);
  else note_bad_combo("lz_combine");
#undef LZC
}

}  // namespace ovl
