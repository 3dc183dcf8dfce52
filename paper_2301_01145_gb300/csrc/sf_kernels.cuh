// sf_kernels.cuh -- kernels of the solver: one-pass launches, the persistent
// work-list executor, and the FP64 set-up kernels for the Green's table.
#pragma once

#include "sf_tiles.cuh"

namespace sfg {

#define SF_THREADS 256
// dynamic shared memory of one general-engine CTA: two CTAs share one SM
#define SF_SMEM_BUDGET (112 * 1024)

// Per-launch pointers: user buffers are kernel arguments so that every launch
// (and every captured graph node) carries its own copy.
template <typename T> struct IOArgs {
  int use;
  int has_face;
  const T *in[SF_MAXF];
  T *out[SF_MAXF];
  const T *face[3][2];
};

template <typename T>
__device__ __forceinline__ void load_prob(Prob<T> &dst, const Prob<T> *src, const IOArgs<T> &io) {
  // cooperative copy of the (read-only) problem description into shared memory
  const int nwords = sizeof(Prob<T>) / 4;
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) d[i] = s[i];
  __syncthreads();
  if (threadIdx.x == 0 && io.use) {
    for (int i = 0; i < SF_MAXF; ++i) {
      dst.in_ptr[i] = io.in[i];
      dst.out_ptr[i] = io.out[i];
    }
    for (int a = 0; a < 3; ++a)
      for (int s2 = 0; s2 < 2; ++s2) dst.face[a][s2] = io.face[a][s2];
    dst.has_face = io.has_face;
  }
  __syncthreads();
}

// one launch = one pass; blockIdx.x is the tile
// Both executors run two CTAs per SM (the shared-memory budget of a pass is
// sized for that), so their register use is held to 65536 / (2 SF_THREADS).
template <typename T>
__global__ void __launch_bounds__(SF_THREADS, 2) k_pass(const Prob<T> *probs, const Pass<T> *passes, int pass_idx, IOArgs<T> io) {
  extern __shared__ __align__(16) unsigned char sf_smem[];
  __shared__ __align__(16) Prob<T> sP;
  __shared__ Pass<T> sPass;
  if (threadIdx.x == 0) sPass = passes[pass_idx];
  __syncthreads();
  load_prob<T>(sP, probs + sPass.prob, io);
  run_tile<T>(sP, sPass, blockIdx.x, reinterpret_cast<cx<T> *>(sf_smem), (size_t)sPass.bufsz);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// release reduction: orders every write this thread has observed (through a
// preceding CTA barrier, the writes of its CTA) before the counter update
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Persistent executor: CTAs pull work items (pass, tile) from a queue in list
// order; an item waits (bounded in time and iterations) until the passes it
// depends on have completed the required number of tiles.  Dependencies only
// point to earlier items, which are held by running CTAs, so progress never
// depends on CTA residency.  A wait that gives up records SF_ERR_TIMEOUT and
// the item is skipped (its counter still advances so nothing else hangs).
template <typename T>
__global__ void __launch_bounds__(SF_THREADS, 2)
    k_exec(const Prob<T> *probs, const Pass<T> *passes, const int *pass_start, int npass, unsigned *done, ExecCtl *ctl,
           unsigned *sticky, unsigned long long timeout_ns, IOArgs<T> io) {
  extern __shared__ __align__(16) unsigned char sf_smem[];
  __shared__ __align__(16) Prob<T> sP;
  __shared__ Pass<T> sPass;
  __shared__ int s_item, s_pass, s_ok, s_prob;
  const int total = pass_start[npass];
  unsigned long long t_wait0 = 0, t_busy0 = 0;  // thread 0: tracing timestamps
  if (threadIdx.x == 0) s_prob = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = (int)atomicAdd(&ctl->next, 1u);
      s_item = it;
      s_ok = 1;
      t_wait0 = global_ns();
      if (it < total) {
        int lo = 0, hi = npass - 1;  // last pass with start <= it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (pass_start[mid] <= it) lo = mid;
          else hi = mid - 1;
        }
        s_pass = lo;
        sPass = passes[lo];
        for (int d = 0; d < 2; ++d) {
          const int dp = sPass.dep[d];
          if (dp < 0) continue;
          const unsigned need = (unsigned)sPass.depcnt[d];
          const unsigned long long t0 = global_ns();
          unsigned iters = 0;
          while (ld_acquire(&done[dp]) < need) {
            __nanosleep(128);
            if (((++iters) & 255u) == 0 && (global_ns() - t0 > timeout_ns || iters > (1u << 28))) {
              atomicCAS(&ctl->error, 0u, 6u);
              atomicExch(&ctl->err_pass, (unsigned)lo);
              atomicOr(sticky, 1u);
              s_ok = 0;
              break;
            }
          }
          if (!s_ok) break;
        }
      }
    }
    if (threadIdx.x == 0 && s_item < total) {
      t_busy0 = global_ns();
      atomicAdd(&ctl->wait_ns[sPass.kind & 7], t_busy0 - t_wait0);
    }
    __syncthreads();
    const int it = s_item;
    if (it >= total) break;
    if (sPass.prob != s_prob) {
      load_prob<T>(sP, probs + sPass.prob, io);
      if (threadIdx.x == 0) s_prob = sPass.prob;
    }
    if (s_ok) run_tile<T>(sP, sPass, it - pass_start[s_pass], reinterpret_cast<cx<T> *>(sf_smem), (size_t)sPass.bufsz);
    __syncthreads();
    if (threadIdx.x == 0) {
      red_release_add(&done[s_pass], 1u);  // publishes the tile (cumulative over the barrier above)
      atomicAdd(&ctl->busy_ns[sPass.kind & 7], global_ns() - t_busy0);
      atomicAdd(&ctl->tiles[sPass.kind & 7], 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 set-up: Green's function octant and its conversion
// ---------------------------------------------------------------------------
// Exponential integral E1(x), x > 0, written from Abramowitz & Stegun:
//   x <= 1:  series 5.1.11, E1 = -gamma - ln x - sum_{k>=1} (-x)^k / (k k!)
//   x >  1:  continued fraction 5.1.22 in its even form
//            E1 = e^-x / (x + 1 - 1/(x + 3 - 4/(x + 5 - 9/(x + 7 - ...)))),
//            evaluated with the modified Lentz method.
__host__ __device__ inline double sf_expint_e1(double x) {
  const double euler = 0.57721566490153286060651209008240243;
  if (x <= 0.0) return 0.0;
  if (x > 700.0) return 0.0;
  if (x <= 1.0) {
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 60; ++k) {
      term *= -x / k;  // (-x)^k / k!
      const double add = term / k;
      sum += add;
      if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return -euler - log(x) - sum;
  }
  const double tiny = 1e-300;
  double b = x + 1.0;
  double c = 1.0 / tiny;
  double d = 1.0 / b;
  double h = d;
  for (int i = 1; i < 500; ++i) {
    const double an = -(double)i * (double)i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// G octant [z][y][x] for offsets 0..n per axis (2D: nz = 0)
// Sine integral Si(x), x >= 0, in FP64 (set-up of the spectral kernel).
//   x <= 4: the power series sum_n (-1)^n x^(2n+1) / ((2n+1) (2n+1)!)  (A&S 5.2.14);
//   x >  4: Si(x) = pi/2 + Im E1(i x), with E1(z) = e^-z / (z + 1 - 1/(z + 3 - 4/(z + 5 - ...)))
//           (the continued fraction of A&S 5.1.22 in even form), evaluated by the
//           modified Lentz method in complex arithmetic (at most 200 terms).
__host__ __device__ inline double sf_sine_integral(double x) {
  const double half_pi = 1.57079632679489661923132169163975144;
  if (x <= 4.0) {
    double p = x, sum = x;  // p = (-1)^n x^(2n+1) / (2n+1)!
    for (int n = 1; n < 40; ++n) {
      p *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
      const double t = p / (2.0 * n + 1.0);
      sum += t;
      if (fabs(t) < 1e-18 * fabs(sum)) break;
    }
    return sum;
  }
  // complex numbers as (re, im) pairs; z = i x
  const double tiny = 1e-300;
  double br = 1.0, bi = x;  // b_1 = z + 1
  double cr = 1.0 / tiny, ci = 0.0;
  double den = br * br + bi * bi;
  double dr = br / den, di = -bi / den;  // d = 1 / b
  double hr = dr, hi = di;
  for (int k = 1; k < 200; ++k) {
    const double a = -(double)k * (double)k;
    br += 2.0;  // b_{k+1} = z + 2k + 1
    // d = 1 / (a d + b)
    double tr = a * dr + br, ti = a * di + bi;
    den = tr * tr + ti * ti;
    dr = tr / den;
    di = -ti / den;
    // c = b + a / c
    den = cr * cr + ci * ci;
    const double qr = a * cr / den, qi = -a * ci / den;
    cr = br + qr;
    ci = bi + qi;
    // h *= c d
    const double er = cr * dr - ci * di, ei = cr * di + ci * dr;
    const double nhr = hr * er - hi * ei, nhi = hr * ei + hi * er;
    hr = nhr;
    hi = nhi;
    if (fabs(er - 1.0) + fabs(ei) < 1e-16) break;
  }
  // E1(ix) = e^{-ix} h
  const double c = cos(x), s = sin(x);
  const double eim = -s * hr + c * hi;  // Im((c - i s)(hr + i hi))
  return half_pi + eim;
}

// ---- double-double arithmetic (Dekker's error-free sum and product) ------
// The error-free steps need each rounded product as such: sf_rmul keeps the
// compiler from fusing it with a following add (nvcc contracts device code,
// and gcc contracts host code on FMA machines).
__host__ __device__ inline double sf_rmul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  volatile double p = a * b;
  return p;
#endif
}
struct sf_dd {
  double hi, lo;
};
__host__ __device__ inline sf_dd sf_dd_two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__host__ __device__ inline sf_dd sf_dd_add(sf_dd a, sf_dd b) {
  sf_dd s = sf_dd_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return sf_dd_two_sum(s.hi, s.lo);
}
__host__ __device__ inline sf_dd sf_dd_mul(sf_dd a, sf_dd b) {
  const double p = sf_rmul(a.hi, b.hi);
  const double e = fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  return sf_dd_two_sum(p, e);
}
__host__ __device__ inline sf_dd sf_dd_div(sf_dd a, double b) {
  const double q1 = a.hi / b;
  const double r = fma(-q1, b, a.hi) + a.lo;  // the remainder a.hi - q1 b is exact
  return sf_dd_two_sum(q1, r / b);
}

// Bessel J0, J1 for x >= 40 from their Hankel asymptotic expansions (A&S 9.2.5,
// 9.2.9, 9.2.10): J_nu(x) = sqrt(2 / (pi x)) [P cos(chi) - Q sin(chi)],
// chi = x - (nu / 2 + 1 / 4) pi, with a_k = prod_{j <= k} (4 nu^2 - (2j - 1)^2) / (k! (8x)^k),
// P = a_0 - a_2 + a_4 - ..., Q = a_1 - a_3 + ...; summed until the terms fall
// below 1e-18 (at x >= 40 they do so long before the series starts to diverge).
__host__ __device__ inline double sf_bessel_j_asym(int nu, double x) {
  const double mu = 4.0 * nu * nu;
  double a = 1.0, P = 1.0, Q = 0.0;
  for (int k = 1; k < 60; ++k) {
    a *= (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (k * 8.0 * x);
    const int r = k & 3;  // signs + (k = 0), + (1), - (2), - (3), + (4) ...
    const double t = (r == 2 || r == 3) ? -a : a;
    if (k & 1) Q += t;
    else P += t;
    if (fabs(a) < 1e-18) break;
  }
  const double pi = 3.14159265358979323846264338327950288;
  const double chi = x - (0.5 * nu + 0.25) * pi;
  return sqrt(2.0 / (pi * x)) * (P * cos(chi) - Q * sin(chi));
}

// F(x) = int_0^x (1 - J0(t)) / t dt, x >= 0, in FP64 (set-up of the 2D
// spectral kernel).
//   x <= 40: the power series sum_{m >= 1} (-1)^(m+1) (x^2/4)^m / (2m (m!)^2)
//            (term-wise integration of J0's series), summed in double-double
//            arithmetic so that its cancellation (terms up to ~1e15 at x = 40)
//            leaves a result accurate to FP64 rounding;
//   x >  40: F(x) = ln(x/2) + gamma + I(x), I(x) = int_x^inf J0(t)/t dt (the
//            limit of F(x) - ln x is gamma - ln 2), with I from repeated
//            integration by parts (J0 = J1' + J1/t, J1 = -J0'):
//            I_n = -J1/x^n + (n+1) J0/x^(n+1) - (n+1)^2 I_(n+2) for
//            I_n = int_x^inf J0(t) t^-n dt, summed until the smallest term.
__host__ __device__ inline double sf_int_1mj0(double x) {
  if (x <= 0.0) return 0.0;
  if (x <= 40.0) {
    const double x2 = sf_rmul(x, x);
    const sf_dd xx = sf_dd_two_sum(x2, fma(x, x, -x2));
    const sf_dd q = {xx.hi * 0.25, xx.lo * 0.25};
    sf_dd term = {1.0, 0.0};  // (x^2/4)^m / (m!)^2
    sf_dd sum = {0.0, 0.0};
    for (int m = 1; m < 200; ++m) {
      term = sf_dd_div(sf_dd_mul(term, q), (double)m * (double)m);
      sf_dd t = sf_dd_div(term, 2.0 * m);
      if (!(m & 1)) {
        t.hi = -t.hi;
        t.lo = -t.lo;
      }
      sum = sf_dd_add(sum, t);
      if ((double)m * (double)m > q.hi && fabs(t.hi) < 1e-20 * fabs(sum.hi)) break;
    }
    return sum.hi + sum.lo;
  }
  const double euler = 0.57721566490153286060651209008240243;
  const double j0 = sf_bessel_j_asym(0, x), j1 = sf_bessel_j_asym(1, x);
  // I_1 = sum_k (-1)^k c_k [-J1 / x^(2k+1) + (2k+2) J0 / x^(2k+2)], c_k = (2^k k!)^2
  double c = 1.0, xp = x, I = 0.0, prev = 1e300;
  for (int k = 0; k < 60; ++k) {
    const double t = c * (-j1 / xp + (2.0 * k + 2.0) * j0 / (xp * x));
    if (fabs(t) > prev) break;  // asymptotic series: stop at its smallest term
    I += (k & 1) ? -t : t;
    prev = fabs(t);
    if (prev < 1e-22) break;
    c *= (2.0 * k + 2.0) * (2.0 * k + 2.0);
    xp *= x * x;
  }
  return log(0.5 * x) + euler + I;
}

// Correction of the order-P kernel over G2 (P = 2m): sigma^2 zeta_sigma(r) Q_m(u),
// u = r^2 / sigma^2, with Q_m = sum_{j=1}^{m-1} p_{j-1}(u) / (2^j j!) and p_j the
// polynomial of (-lap)^j zeta_sigma = zeta_sigma p_j(u) / sigma^{2j} in d
// dimensions (p_0 = 1; 3D p_1 = 3 - u, p_2 = u^2 - 10u + 15, p_3 = -u^3 + 21u^2 -
// 105u + 105; 2D p_1 = 2 - u, p_2 = u^2 - 8u + 8, p_3 = -u^3 + 18u^2 - 72u + 48).
// Coefficients of Q_m in powers of u, m = 2..5:
__device__ __forceinline__ double kernel_q(int dim, int m, double u) {
  if (m <= 1) return 0.0;
  if (dim == 3) {
    switch (m) {
      case 2: return 0.5;
      case 3: return 7.0 / 8.0 - u / 8.0;
      case 4: return 19.0 / 16.0 - u / 3.0 + u * u / 48.0;
      default: return 187.0 / 128.0 - 233.0 * u / 384.0 + 29.0 * u * u / 384.0 - u * u * u / 384.0;
    }
  }
  switch (m) {
    case 2: return 0.5;
    case 3: return 0.75 - u / 8.0;
    case 4: return 11.0 / 12.0 - 7.0 * u / 24.0 + u * u / 48.0;
    default: return 25.0 / 24.0 - 23.0 * u / 48.0 + 13.0 * u * u / 192.0 - u * u * u / 384.0;
  }
}

// order: 2..10 for the Gaussian kernels (2D, 3D), 0 for the spectral cut-off at kc (1D, 3D)
static __global__ void k_green_octant(double *out, int nx, int ny, int nz, double hx, double hy, double hz, double sigma,
                               int dim, int order, double kc) {
  const size_t total = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const double pi = 3.14159265358979323846264338327950288;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % (nx + 1));
    const size_t r1 = i / (nx + 1);
    const int y = (int)(r1 % (ny + 1));
    const int z = (int)(r1 / (ny + 1));
    const double dx = x * hx, dy = y * hy, dz = z * hz;
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double g;
    if (order == 0 && dim == 1) {  // spectral, 1D: -(r Si(kc r) + cos(kc r) / kc) / pi
      g = -(r * sf_sine_integral(kc * r) + cos(kc * r) / kc) / pi;
    } else if (order == 0 && dim == 2) {  // spectral, 2D: (ln(kc/2) + gamma - F(kc r)) / (2 pi)
      const double euler = 0.57721566490153286060651209008240243;
      g = (log(0.5 * kc) + euler - sf_int_1mj0(kc * r)) / (2.0 * pi);
    } else if (order == 0) {  // spectral, 3D: Si(kc r) / (2 pi^2 r)
      g = r == 0.0 ? kc / (2.0 * pi * pi) : sf_sine_integral(kc * r) / (2.0 * pi * pi * r);
    } else if (dim == 3) {
      if (r == 0.0) g = sqrt(2.0) / (4.0 * pi * sqrt(pi) * sigma);
      else g = erf(r / (sigma * sqrt(2.0))) / (4.0 * pi * r);
    } else {
      const double euler = 0.57721566490153286060651209008240243;
      if (r == 0.0) g = (0.5 * euler - log(sqrt(2.0) * sigma)) / (2.0 * pi);
      else g = -(log(r) + 0.5 * sf_expint_e1(r * r / (2.0 * sigma * sigma))) / (2.0 * pi);
    }
    if (order > 2) {  // higher-order Gaussian kernel: G2 + sigma^2 zeta_sigma(r) Q_m(u)
      const double u = r * r / (sigma * sigma);
      const double zeta = exp(-0.5 * u) / (dim == 3 ? pow(2.0 * pi * sigma * sigma, 1.5) : 2.0 * pi * sigma * sigma);
      g += sigma * sigma * zeta * kernel_q(dim, order / 2, u);
    }
    out[i] = g;
  }
}

// Semi-unbounded Green's table, one CTA per periodic mode (row): the kernel row
// g[m] = exp(-kappa m h) / (2 kappa) (kappa > 0) or -m h / 2 (kappa = 0) for the
// offsets m = 0 .. Lu/2 of the doubled unbounded axis, then its DCT-I
// g[0] + (-1)^k g[Lu/2] + 2 sum_{0 < m < Lu/2} g[m] cos(2 pi k m / Lu) at every
// k = 0 .. Lu/2 (the DFT of the mirrored row).  The table is laid out like the
// all-unbounded one: [i0][i2][i1] in 3D, [i0][i1] in 2D, with the unbounded
// axis's index k and the periodic indices of the row (row = i_pa * eb + i_pb).
static __global__ void k_green_semi(double *out, const double *kap2, int dim, int ua, int pa, int pb, int e0, int e1,
                                    int e2, int eb, int Lu, double hu) {
  extern __shared__ double gsem[];
  double *cs = gsem;       // cos(2 pi j / Lu), j < Lu
  double *g = gsem + Lu;   // kernel row, m <= Lu / 2
  const int half = Lu / 2;
  const int row = blockIdx.x;
  const double k2 = kap2[row];
  const double kap = k2 > 0.0 ? sqrt(k2) : 0.0;
  for (int j = threadIdx.x; j < Lu; j += blockDim.x) cs[j] = cospi(2.0 * j / Lu);
  for (int m = threadIdx.x; m <= half; m += blockDim.x) {
    const double z = m * hu;
    g[m] = kap > 0.0 ? exp(-kap * z) / (2.0 * kap) : -0.5 * z;
  }
  __syncthreads();
  int c[3] = {0, 0, 0};
  c[pa] = row / eb;
  if (pb >= 0) c[pb] = row % eb;
  for (int k = threadIdx.x; k <= half; k += blockDim.x) {
    double acc = 0.0;
    int idx = 0;  // k m mod Lu
    for (int m = 1; m < half; ++m) {
      idx += k;
      if (idx >= Lu) idx -= Lu;
      acc += g[m] * cs[idx];
    }
    const double v = g[0] + ((k & 1) ? -g[half] : g[half]) + 2.0 * acc;
    c[ua] = k;
    const size_t o = dim == 3 ? ((size_t)c[0] * e2 + c[2]) * e1 + c[1] : (size_t)c[0] * e1 + c[1];
    out[o] = v;
  }
}

// [kx][kz][ky] -> [kx][ky][kz] (set-up only)
template <typename T> __global__ void k_transpose_green(T *out, const T *in, int nkx, int nkz, int nky) {
  const size_t total = (size_t)nkx * nkz * nky;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(i % nky);
    const size_t r = i / nky;
    const int kz = (int)(r % nkz);
    const int kx = (int)(r / nkz);
    out[((size_t)kx * nky + ky) * nkz + kz] = in[i];
  }
}

template <typename T> __global__ void k_convert_scale(T *out, const double *in, size_t n, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)(in[i] * scale);
}

}  // namespace sfg
