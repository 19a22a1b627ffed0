// Multi-shift conjugate gradient for the Zolotarev sign function (Sec. 3):
// all shifted systems (K^2 + sigma_i) x_i = v, i = 1..N_Z, share the Krylov
// space of the base system K^2 + sigma_0 (sigma_0 the smallest shift), and only
// y = sum_i omega_i x_i is kept. Every scalar of the recurrence stays on the
// device, so a whole step is five launches with no host round trip:
//
//   wilson MODE_K   t = K p_0, partials ||t||^2, ||p_0||^2
//   ms_scalar1      alpha = rr / (||t||^2 + sigma0 ||p_0||^2); zeta_{k+1}, alpha_i
//   wilson MODE_R   r -= alpha (K t + sigma0 p_0), partials ||r||^2
//   ms_scalar2      beta, beta_i, pole dropping, done flag
//   ms_update       y += sum_i omega_i alpha_i p_i ; p_i = zeta_i r + beta_i p_i
//
// Stopping rule (the reading of "eta = Delta or the error in the inversion of
// x^2 + sigma_i, whichever is larger"): pole i contributes at most
// e_i = omega_i g_i |zeta_i| ||r|| to the error of eps(K) v, with
// g_i = max_{a<=x<=b} x/(x^2+sigma_i), and the solve may end once the e_i of the
// running poles and those frozen by the stopped ones sum to eta ||v||; poles drop
// from the largest shift down (they converge first). See ms_scalar2_kernel for how
// the budget is shared.
#include "kernels.h"

namespace ovl {

// ---------------------------------------------------------------- init
template <int PV, int PR, int PP>
__global__ void __launch_bounds__(256) ms_init_kernel(SpinorRef v, SpinorRef r, SpinorRef pb, SpinorRef y,
                                                      int npoles, int nrhs, int V, int nsb, int ngr,
                                                      double* partials) {
  using T = typename Real<PR>::T;
  __shared__ double red[4 * (BX / 32) * 2];
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (s < V && rhs < nrhs) {
    cpx<T> a[12], z[12];
    load_spinor_as<PV, T>(v, rhs, s, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[0] += (double)norm2(a[k]);
      z[k] = cmk(T(0), T(0));
    }
    store_spinor_as<PR, T>(r, rhs, s, a);
    store_spinor_as<PR, T>(y, rhs, s, z);
    for (int i = 0; i < npoles; ++i) store_spinor_as<PP, T>(pb, i * nrhs + rhs, s, a);
  }
  block_reduce_rows<2>(acc, red);
  if (threadIdx.x == 0 && rhs < nrhs) {
    partials[((size_t)rhs * nsb + sb) * NVRED + 0] = acc[0];
    partials[((size_t)rhs * nsb + sb) * NVRED + 1] = 0.0;
  }
}

void launch_ms_init(int pv, int pr, int pp, SpinorRef v, SpinorRef r, SpinorRef pb, SpinorRef y, int npoles,
                    int nrhs, int V, double* partials, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
#define MS_INIT(A, B, C) ms_init_kernel<A, B, C><<<sh.grid(), sh.block(), 0, st>>>(v, r, pb, y, npoles, nrhs, V, sh.nsb, sh.ngr, partials)
  if (pv == P64 && pr == P64 && pp == P64) MS_INIT(P64, P64, P64);
  else if (pv == P32 && pr == P32 && pp == P32) MS_INIT(P32, P32, P32);
  else if (pv == P64 && pr == P32 && pp == P32) MS_INIT(P64, P32, P32);
  else if (pv == P32 && pr == P32 && pp == P16) MS_INIT(P32, P32, P16);
  else if (pv == P64 && pr == P32 && pp == P16) MS_INIT(P64, P32, P16);
  else if (pv == P32 && pr == P64 && pp == P64) MS_INIT(P32, P64, P64);
  else if (pv == P64 && pr == P64E && pp == P64E) MS_INIT(P64, P64E, P64E);
  else if (pv == P32 && pr == P64E && pp == P64E) MS_INIT(P32, P64E, P64E);
  else note_bad_combo("ms_init");
#undef MS_INIT
}

// ---------------------------------------------------------------- scalars
// Fixed-order sum of the NVRED-wide partials of one rhs by one block.
__device__ __forceinline__ void sum_partials(const double* partials, int nsb, int rhs, double out[2]) {
  __shared__ double sh[2][128];
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < nsb; b += blockDim.x) {
    a0 += partials[((size_t)rhs * nsb + b) * NVRED + 0];
    a1 += partials[((size_t)rhs * nsb + b) * NVRED + 1];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  out[0] = sh[0][0];
  out[1] = sh[1][0];
  __syncthreads();
}

__global__ void ms_scalar0_kernel(MsRhs* ms, const double* partials, int nsb, const Poles* P, const double* eta,
                                  int maxit) {
  const int rhs = blockIdx.x;
  double s[2];
  sum_partials(partials, nsb, rhs, s);
  MsRhs& m = ms[rhs];
  for (int i = threadIdx.x; i < NPMAX; i += blockDim.x) {
    m.zeta[i] = 1.0;
    m.zeta_prev[i] = 1.0;
    m.zeta_next[i] = 1.0;
    m.coef_y[i] = 0.0;
    m.coef_r[i] = 0.0;
    m.coef_p[i] = 0.0;
    m.coef_a[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    m.rr = s[0];
    m.consumed = 0.0;
    m.alpha = 0.0;
    m.alpha_prev = 1.0;
    m.beta_prev = 0.0;
    // per-pole share of the error budget |eta| ||v||; the sign of eta (set by the host)
    // selects the stopping rule: positive, one budget shared by all poles; negative,
    // every pole within its even share
    m.thr = eta[rhs] * sqrt(s[0]) / (double)P->n;
    m.active = P->n;
    m.nact_y = 0;
    m.iter = 0;
    m.maxit = maxit;
    m.status = 0;
    m.p_reads = 0;
    m.p_writes = 0;
    m.done = (s[0] == 0.0) ? 1 : 0;
  }
}

__global__ void ms_scalar1_kernel(MsRhs* ms, const double* partials, int nsb, const Poles* P) {
  const int rhs = blockIdx.x;
  MsRhs& m = ms[rhs];
  if (m.done) return;
  double s[2];
  sum_partials(partials, nsb, rhs, s);
  const double pAp = s[0] + P->sigma0 * s[1];
  const double alpha = m.rr / pAp;
  const bool bad = !(pAp > 0.0) || !isfinite(alpha);
  for (int i = threadIdx.x; i < m.active; i += blockDim.x) {
    const double z = m.zeta[i], zp = m.zeta_prev[i];
    double zn = 0.0, as = 0.0;
    if (z != 0.0) {
      const double den = alpha * m.beta_prev * (zp - z) + zp * m.alpha_prev * (1.0 + P->ds[i] * alpha);
      zn = z * zp * m.alpha_prev / den;
      as = alpha * zn / z;
    }
    m.zeta_next[i] = zn;
    m.coef_y[i] = P->omega[i] * as;
    m.coef_a[i] = as;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    m.alpha = alpha;
    if (bad) {
      m.done = 1;
      m.status = 2;   // breakdown
      m.nact_y = 0;
    }
  }
}

__global__ void ms_scalar2_kernel(MsRhs* ms, const double* partials, int nsb, const Poles* P) {
  const int rhs = blockIdx.x;
  MsRhs& m = ms[rhs];
  if (m.done) {
    if (threadIdx.x == 0) m.nact_y = 0;
    return;
  }
  double s[2];
  sum_partials(partials, nsb, rhs, s);
  const double rr_new = s[0];
  const double beta = rr_new / m.rr;
  const int act = m.active;
  for (int i = threadIdx.x; i < act; i += blockDim.x) {
    const double z = m.zeta[i], zn = m.zeta_next[i];
    const double q = (z != 0.0) ? zn / z : 0.0;
    m.coef_r[i] = zn;
    m.coef_p[i] = beta * q * q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    m.nact_y = act;
    const double rn = sqrt(rr_new);
    // Error bound of pole i if stopped now: omega_i g_i |zeta_i| ||r||; the sign is within
    // eta ||v|| = N |thr| once the bounds of the stopped and the running poles add up to
    // less. Accurate signs: shifted poles (largest sigma first) stop at a quarter of the
    // even share, which saves their update passes, and the system stops as soon as the
    // sum of all bounds is within the whole budget, so the slowest (base) pole uses what
    // the others left. Even shares (relaxed signs of relCG): every pole within thr,
    // which keeps the actual sign error well below the relaxation's eta_j.
    auto bound = [&](int i) { return P->omega[i] * P->gbound[i] * fabs(m.zeta_next[i]) * rn; };
    int a = act;
    if (m.thr > 0.0) {
      while (a > 1 && bound(a - 1) <= 0.25 * m.thr) {
        m.consumed += bound(a - 1);
        --a;
      }
      double tot = m.consumed;
      for (int i = 0; i < a; ++i) tot += bound(i);
      if (tot <= m.thr * (double)P->n) {
        m.consumed = tot;
        a = 0;
      }
    } else {
      while (a > 0 && bound(a - 1) <= -m.thr) --a;
    }
    m.active = a;
    m.p_reads += act;
    m.p_writes += a;
    m.alpha_prev = m.alpha;
    m.beta_prev = beta;
    m.rr = rr_new;
    m.iter += 1;
    if (!isfinite(rr_new)) {
      m.done = 1;
      m.status = 2;
    } else if (a == 0) {
      m.done = 1;
      m.status = 0;
    } else if (m.iter >= m.maxit) {
      m.done = 1;
      m.status = 1;   // not converged
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < act; i += blockDim.x) {
    m.zeta_prev[i] = m.zeta[i];
    m.zeta[i] = m.zeta_next[i];
  }
}

void launch_ms_scalar0(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles, const double* eta,
                       int maxit, cudaStream_t st) {
  ms_scalar0_kernel<<<nrhs, 128, 0, st>>>(ms, partials, nsb, poles, eta, maxit);
}
void launch_ms_scalar1(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles, cudaStream_t st) {
  ms_scalar1_kernel<<<nrhs, 128, 0, st>>>(ms, partials, nsb, poles);
}
void launch_ms_scalar2(MsRhs* ms, const double* partials, int nsb, int nrhs, const Poles* poles, cudaStream_t st) {
  ms_scalar2_kernel<<<nrhs, 128, 0, st>>>(ms, partials, nsb, poles);
}

// ---------------------------------------------------------------- fused update
// One pass over every active pole vector: y += omega_i alpha_i p_i (old p_i), then
// p_i = zeta_{k+1,i} r + beta_i p_i. Pole 0 is the base system (zeta = 1).
template <int PR, int PP>
__global__ void __launch_bounds__(256) ms_update_kernel(SpinorRef r, SpinorRef pb, SpinorRef y, int npoles,
                                                        int nrhs, int V, int ngr, const MsRhs* ms) {
  using T = typename Real<PR>::T;
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  if (s >= V || rhs >= nrhs) return;
  const MsRhs& m = ms[rhs];
  const int ny = m.nact_y;
  if (ny == 0) return;
  const int na = m.active;
  cpx<T> rv[12], yv[12], pv[12];
  load_spinor_as<PR, T>(r, rhs, s, rv);
  load_spinor_as<PR, T>(y, rhs, s, yv);
  for (int i = 0; i < ny; ++i) {
    load_spinor_as<PP, T>(pb, i * nrhs + rhs, s, pv);
    const T cy = (T)m.coef_y[i];
#pragma unroll
    for (int k = 0; k < 12; ++k) yv[k] = yv[k] + cy * pv[k];
    if (i < na) {
      const T cr = (T)m.coef_r[i], cp = (T)m.coef_p[i];
#pragma unroll
      for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
      store_spinor_as<PP, T>(pb, i * nrhs + rhs, s, pv);
    }
  }
  store_spinor_as<PR, T>(y, rhs, s, yv);
}

// Double-float form of the same pass, chunk-major: for each 16-byte chunk (one complex
// component) of r and y, every active pole's chunk is read, y accumulated and the pole
// rewritten. Holding one component instead of whole spinors keeps the thread small
// (the spinor-at-a-time form needs ~250 registers: 8 warps per SM, 78% of the copy
// bandwidth), and the pole coefficients are converted to double-float once per block
// into shared memory instead of per thread and pole.
__global__ void __launch_bounds__(256) ms_update_df_kernel(SpinorRef r, SpinorRef pb, SpinorRef y, int nrhs, int V,
                                                           int ngr, const MsRhs* ms) {
  __shared__ float2 cf[4][NPMAX][3];   // (y, r, p) coefficients of the block's systems
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const bool in_rhs = rhs < nrhs;
  const int ny = in_rhs ? ms[rhs].nact_y : 0;
  if (in_rhs) {
    const MsRhs& m = ms[rhs];
    for (int i = threadIdx.x; i < ny; i += blockDim.x) {
      const double c3[3] = {m.coef_y[i], m.coef_r[i], m.coef_p[i]};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float h = (float)c3[k];
        cf[threadIdx.y][i][k] = make_float2(h, (float)(c3[k] - (double)h));
      }
    }
  }
  __syncthreads();
  const int s = sb * BX + threadIdx.x;
  if (s >= V || !in_rhs || ny == 0) return;
  const int na = ms[rhs].active;
  const size_t Vs = (size_t)V;
  const float4* rr = reinterpret_cast<const float4*>(r.data) + (size_t)rhs * 12 * Vs + s;
  float4* yy = reinterpret_cast<float4*>(y.data) + (size_t)rhs * 12 * Vs + s;
  float4* pp = reinterpret_cast<float4*>(pb.data) + (size_t)rhs * 12 * Vs + s;
  const size_t pole_stride = (size_t)nrhs * 12 * Vs;
  const float2(*c)[3] = cf[threadIdx.y];
  for (int k = 0; k < 12; ++k) {
    const float4 rw = rr[(size_t)k * Vs];
    const cpx<df> rc = cmk(df(rw.x, rw.y), df(rw.z, rw.w));
    const float4 yw = yy[(size_t)k * Vs];
    cpx<df> yc = cmk(df(yw.x, yw.y), df(yw.z, yw.w));
    for (int i = 0; i < ny; ++i) {
      float4* pi = pp + (size_t)i * pole_stride + (size_t)k * Vs;
      const float4 pw = *pi;
      cpx<df> pc = cmk(df(pw.x, pw.y), df(pw.z, pw.w));
      const df cy(c[i][0].x, c[i][0].y);
      yc = yc + cy * pc;
      if (i < na) {
        const df cr(c[i][1].x, c[i][1].y), cp(c[i][2].x, c[i][2].y);
        pc = cr * rc + cp * pc;
        *pi = make_float4(pc.r.hi, pc.r.lo, pc.i.hi, pc.i.lo);
      }
    }
    yy[(size_t)k * Vs] = make_float4(yc.r.hi, yc.r.lo, yc.i.hi, yc.i.lo);
  }
}

void launch_ms_update(int pr, int pp, SpinorRef r, SpinorRef pb, SpinorRef y, int npoles, int nrhs, int V,
                      const MsRhs* ms, cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  if (pr == P64E && pp == P64E) {
    ms_update_df_kernel<<<sh.grid(), sh.block(), 0, st>>>(r, pb, y, nrhs, V, sh.ngr, ms);
    return;
  }
  if (pr == P64 && pp == P64) ms_update_kernel<P64, P64><<<sh.grid(), sh.block(), 0, st>>>(r, pb, y, npoles, nrhs, V, sh.ngr, ms);
  else if (pr == P32 && pp == P32) ms_update_kernel<P32, P32><<<sh.grid(), sh.block(), 0, st>>>(r, pb, y, npoles, nrhs, V, sh.ngr, ms);
  else if (pr == P32 && pp == P16) ms_update_kernel<P32, P16><<<sh.grid(), sh.block(), 0, st>>>(r, pb, y, npoles, nrhs, V, sh.ngr, ms);
  else note_bad_combo("ms_update");
}

}  // namespace ovl

namespace ovl {
__global__ void __launch_bounds__(256) ms_update_x_kernel(SpinorRef r, SpinorRef pb, SpinorRef xs, int npoles,
                                                          int nrhs, int V, int ngr, const MsRhs* ms) {
  const int sb = blockIdx.x / ngr;
  const int rg = blockIdx.x - sb * ngr;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const int s = sb * BX + threadIdx.x;
  if (s >= V || rhs >= nrhs) return;
  const MsRhs& m = ms[rhs];
  const int ny = m.nact_y;
  if (ny == 0) return;
  const int na = m.active;
  cpx<double> rv[12], xv[12], pv[12];
  load_spinor<P64, double>(r, rhs, s, rv);
  for (int i = 0; i < ny; ++i) {
    load_spinor<P64, double>(pb, i * nrhs + rhs, s, pv);
    load_spinor<P64, double>(xs, i * nrhs + rhs, s, xv);
    const double ca = m.coef_a[i];
#pragma unroll
    for (int k = 0; k < 12; ++k) xv[k] = xv[k] + ca * pv[k];
    store_spinor<P64, double>(xs, i * nrhs + rhs, s, xv);
    if (i < na) {
      const double cr = m.coef_r[i], cp = m.coef_p[i];
#pragma unroll
      for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
      store_spinor<P64, double>(pb, i * nrhs + rhs, s, pv);
    }
  }
}
void launch_ms_update_x(SpinorRef r, SpinorRef pb, SpinorRef xs, int npoles, int nrhs, int V, const MsRhs* ms,
                        cudaStream_t st) {
  Shape sh = make_shape(V, nrhs);
  ms_update_x_kernel<<<sh.grid(), sh.block(), 0, st>>>(r, pb, xs, npoles, nrhs, V, sh.ngr, ms);
}
}  // namespace ovl
