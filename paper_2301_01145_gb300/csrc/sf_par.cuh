// sf_par.cuh -- parity-split y / z stages of the register fast path for the
// zero-padded (unbounded, Hockney-Eastwood) 512-point axes of the 3D curl solve.
//
// A 512-point DFT of a line that is zero in its upper half (Sec. 2.6: the
// source occupies the first N = 256 points of the doubled axis) splits by the
// parity p of the output index k = 2m + p into two 256-point DFTs:
//   X[2m + p] = sum_{n < 256} x[n] W_512^{n (2m + p)},
// and the inverse restricted to the first 256 outputs is the sum of the two
// parity parts y_p[n] = W_512^{-n p} sum_m X[2m + p] W_256^{-n m}.  The zero
// half costs nothing and no lane shuffles are needed.  Spectral rows are kept
// in parity-major order k' = 256 p + m.
//
// Each 256-point transform is a four-step 16 x 16 split, n = u + 16 s,
// m = k1 + 16 k2:
//   stage 1 (fixed u):  a_s = x[u + 16 s] W_32^{s p};  Y[k1] = DFT16_s(a)[k1] * W_512^{u (2 k1 + p)}
//   stage 2 (fixed k1): X_p[k1 + 16 k2] = DFT16_u(Y_u[k1])[k2]
// and the inverse runs the two stages transposed (conjugate twiddles).  The
// exchange between the stages goes through shared memory for a whole tile of
// lines at once, and the thread arrangement of each stage is chosen so that
// this exchange is also the layout change between the passes: loads and
// stores of the intermediate rows are contiguous 128-byte (64-byte for the
// z stage's 8-line tiles) segments and no separate staging transpose is made.
//
//   YF  rows of A [c][kx][z][y] along y  -> I1 [c][kxl][k'y][z]
//   ZS  rows of I1 along z: forward, Green's multiply, d/dz, inverse, sum of
//       the z parities                   -> I2 [f][kxl][z][k'y]  (f: psi_x,y,z, d/dz psi_x,y)
//   YI  rows of I2 along k'y, the curl formed in y-spectral space, inverse,
//       sum of the y parities            -> B  [f][kx][z][y]
// A and B are the same arrays as in the other fast-path variants (natural kx,
// y and z order), so the x transforms are unchanged.
#pragma once

#include "sf_device.cuh"

namespace sfg {

// parity twiddle tables appended to Axis::twf of a 512-point axis (complex entries):
//   twf[SF_TWP_OFF + 256 p + 16 k1 + u]       = W_512^{u (2 k1 + p)}   (forward stage 1: row k1, lane u)
//   twf[SF_TWP_OFF + 512 + 256 p + 16 u + k1] = W_512^{u (2 k1 + p)}   (inverse stage 1: row u, thread k1)
#define SF_TWP_OFF 576
#define SF_PAR_THREADS 256  // threads per CTA of every parity tile

// a * W_32^{-+s} for a compile-time s (forward: W = exp(-2 pi i s / 32); inverse: its conjugate)
template <bool INV> __device__ __forceinline__ float2 w32mul(float2 a, int s) {
  if (s == 0) return a;
  if (s == 8) return mul_mi<INV>(a);
  if (s == 4) return w8<INV>(a, 1);
  if (s == 12) return w8<INV>(a, 3);
  const float2 w = w32c<float2>(s);
  return INV ? cmulc(a, w) : cmul(a, w);
}

// forward stage 1 of parity P on v[s] = x[u + 16 s]; leaves Y[k1] (twiddled) in v[k1]
template <int P> __device__ __forceinline__ void par_fwd1(float2 (&v)[16], const float2 *__restrict__ twp, int u) {
  if (P) {
#pragma unroll
    for (int s = 1; s < 16; ++s) v[s] = w32mul<false>(v[s], s);
  }
  dft16<false>(v);
#pragma unroll
  for (int k1 = P ? 0 : 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], __ldg(&twp[256 * P + 16 * k1 + u]));
}

// inverse stage 1 of parity P for thread k1 on v[k2] = X_P[k1 + 16 k2]; leaves Z_k1[u] in v[u]
template <int P> __device__ __forceinline__ void par_inv1(float2 (&v)[16], const float2 *__restrict__ twp, int k1) {
  dft16<true>(v);
#pragma unroll
  for (int u = P ? 0 : 1; u < 16; ++u) v[u] = cmulc(v[u], __ldg(&twp[512 + 256 * P + 16 * u + k1]));
}

// inverse stage 2 of parity P for thread u on v[k1] = Z_k1[u]; leaves y_P[u + 16 s] in v[s]
template <int P> __device__ __forceinline__ void par_inv2(float2 (&v)[16]) {
  dft16<true>(v);
  if (P) {
#pragma unroll
    for (int s = 1; s < 16; ++s) v[s] = w32mul<true>(v[s], s);
  }
}

// signed FFT index of the parity-major spectral position (p, m) on a 512-point
// axis, as a float multiple of the axis's wavenumber unit; 0 at Nyquist (k = 256)
__device__ __forceinline__ float par_kap(int p, int m, float kap1) {
  const int k = 2 * m + p;
  const int ks = k < 256 ? k : (k > 256 ? k - 512 : 0);
  return (float)ks * kap1;
}

// tile geometry (shared by the host pass lists)
#define SF_PAR_YF_ROWS 16  // z rows per YF tile
#define SF_PAR_ZS_ROWS 8   // k'y rows per ZS tile
#define SF_PAR_YI_ROWS 16  // z rows per YI tile
#define SF_PAR_LS16 273    // line stride (complex) of a 16-line exchange buffer (odd: conflict-free)
#define SF_PAR_LS8 274     // line stride of an 8-line exchange buffer (2 mod 16)

// shared memory of the parity tiles (bytes): the larger of YF / YI (two
// parities x 16 lines) and ZS (two outputs x two parities x 8 lines)
__host__ __device__ constexpr int par_ex16_elems() { return 2 * 16 * SF_PAR_LS16; }
__host__ __device__ constexpr int par_zs_ex_elems() { return 2 * 2 * SF_PAR_ZS_ROWS * SF_PAR_LS8; }
__host__ __device__ constexpr size_t par_smem_bytes() {
  return (size_t)(par_zs_ex_elems() > par_ex16_elems() ? par_zs_ex_elems() : par_ex16_elems()) * 8;
}

// ---------------------------------------------------------------------------
// YF: 16 z rows (fixed c, kx) of A along y, both y parities -> I1 [c][kxl][k'y][z]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void par_yf(const Prob<float> &P, int S, size_t slot_off, int kx0, int nkx, int tile,
                                       float2 *X) {
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, SF_PAR_YF_ROWS);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % nkx;
  const int c = rest / nkx;
  if (c >= P.nin) return;  // uniform over the block
  const int kx = kx0 + kxl;
  const int z0 = iz * SF_PAR_YF_ROWS;
  const float2 *twp = P.ax[1].twf + SF_TWP_OFF;
  {
    // stage 1: half-warp hw transforms row z0 + hw (lane u holds y = u + 16 s)
    const int hw = threadIdx.x >> 4, u = threadIdx.x & 15;
    const int z = z0 + hw;
    const float2 *src = reinterpret_cast<const float2 *>(P.A) + (((size_t)c * nsx + kx) * nuz + z) * nuy;
    float2 a[16], b[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int y = u + 16 * s;
      a[s] = (z < nuz && y < nuy) ? __ldcs(&src[y]) : czero<float2>();
      b[s] = a[s];
    }
    par_fwd1<0>(a, twp, u);
    par_fwd1<1>(b, twp, u);
    float2 *x0 = X + hw * SF_PAR_LS16 + u;
    float2 *x1 = x0 + 16 * SF_PAR_LS16;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
      x0[17 * k1] = a[k1];
      x1[17 * k1] = b[k1];
    }
  }
  __syncthreads();
  {
    // stage 2: thread (k1, zl), z fastest, both parities; rows of I1 stored along z
    const int zl = threadIdx.x & 15, k1 = threadIdx.x >> 4;
    float2 *I1 = reinterpret_cast<float2 *>(P.I1) + slot_off + (((size_t)c * S + kxl) * 512) * nuz;
    const bool ok = z0 + zl < nuz;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float2 v[16];
      const float2 *xs = X + (p * 16 + zl) * SF_PAR_LS16 + 17 * k1;
#pragma unroll
      for (int uu = 0; uu < 16; ++uu) v[uu] = xs[uu];
      dft16<false>(v);
      if (ok) {
        float2 *dst = I1 + (size_t)(256 * p + k1) * nuz + z0 + zl;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) __stcg(&dst[(size_t)16 * k2 * nuz], v[k2]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// ZS: 8 k'y rows (fixed c, kx) of I1 along z: both z parities forward,
// Green's multiply, d/dz (c = x, y), inverse, sum of the parities -> I2
// [f][kxl][z][k'y] (f = c: psi_c, f = 3 + c: d/dz psi_c)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void par_zs(const Prob<float> &P, int S, size_t slot_off, int kx0, int nkx, int tile,
                                       float2 *X) {
  const int nuz = P.nuz;
  constexpr int NTY = 512 / SF_PAR_ZS_ROWS;
  const int iy = tile % NTY;
  const int rest = tile / NTY;
  const int kxl = rest % nkx;
  const int c = rest / nkx;
  if (c >= 3) return;  // uniform over the block
  const int kx = kx0 + kxl;
  const int ky0 = iy * SF_PAR_ZS_ROWS;
  const float2 *twp = P.ax[2].twf + SF_TWP_OFF;
  const float2 *I1 = reinterpret_cast<const float2 *>(P.I1) + slot_off + (((size_t)c * S + kxl) * 512) * nuz;
  // the Green's values this thread multiplies in stage 2 (thread (k1, l, pz)),
  // loaded first so that their latency (the table is mostly not in L2)
  // overlaps stage 1
  float gv[16];
  {
    const int k1 = threadIdx.x & 15, l = (threadIdx.x >> 4) & 7, pz = threadIdx.x >> 7;
    const int lo = 2 * k1 + pz, hi = 512 - 2 * k1 - pz;
    const int kyp = ky0 + l;
    const int ky = 2 * (kyp & 255) + (kyp >> 8);
    const float *g = P.ghat_t + ((size_t)kx * P.gny + min(ky, 512 - ky)) * P.gnz;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) gv[k2] = __ldg(&g[k2 < 8 ? lo + 32 * k2 : hi - 32 * k2]);
  }
  {
    // stage 1: warp-uniform parity pz = warp / 4; half-warp line l
    const int warp = threadIdx.x >> 5, u = threadIdx.x & 15;
    const int pz = warp >> 2;
    const int l = ((warp & 3) << 1) | ((threadIdx.x >> 4) & 1);
    const float2 *src = I1 + (size_t)(ky0 + l) * nuz;
    float2 v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int z = u + 16 * s;
      v[s] = z < nuz ? __ldcg(&src[z]) : czero<float2>();
    }
    if (pz) par_fwd1<1>(v, twp, u);
    else par_fwd1<0>(v, twp, u);
    float2 *xd = X + (pz * SF_PAR_ZS_ROWS + l) * SF_PAR_LS8 + u;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) xd[17 * k1] = v[k1];
  }
  __syncthreads();
  // stage 2 + multiply + inverse stage 1: thread (k1, l, pz), k1 fastest
  const int k1 = threadIdx.x & 15, l = (threadIdx.x >> 4) & 7, pz = threadIdx.x >> 7;
  float2 v[16];
  {
    const float2 *xs = X + (pz * SF_PAR_ZS_ROWS + l) * SF_PAR_LS8 + 17 * k1;
#pragma unroll
    for (int uu = 0; uu < 16; ++uu) v[uu] = xs[uu];
  }
  __syncthreads();  // the exchange buffer is rewritten below
  dft16<false>(v);
  // times the Green's table at kz = 2 (k1 + 16 k2) + pz, folded to min(kz, 512 - kz)
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) v[k2] = cscale(v[k2], gv[k2]);
  if (c < 2) {
    const float kz1 = __ldg(&P.ax[2].kap[1]);
    float2 d[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      // signed index 2 k1 + pz + 32 k2 (- 512 past Nyquist); Nyquist itself (k2 = 8, k1 = pz = 0) gives 0
      float ks = (float)(2 * k1 + pz + 32 * k2 - (k2 >= 8 ? 512 : 0));
      if (k2 == 8 && k1 == 0 && pz == 0) ks = 0.f;
      d[k2] = mul_i(cscale(v[k2], ks * kz1));
    }
    if (pz) par_inv1<1>(d, twp, k1);
    else par_inv1<0>(d, twp, k1);
    float2 *xd = X + ((2 + pz) * SF_PAR_ZS_ROWS + l) * SF_PAR_LS8 + k1;
#pragma unroll
    for (int uu = 0; uu < 16; ++uu) xd[17 * uu] = d[uu];
  }
  if (pz) par_inv1<1>(v, twp, k1);
  else par_inv1<0>(v, twp, k1);
  {
    float2 *xd = X + (pz * SF_PAR_ZS_ROWS + l) * SF_PAR_LS8 + k1;
#pragma unroll
    for (int uu = 0; uu < 16; ++uu) xd[17 * uu] = v[uu];
  }
  __syncthreads();
  if (c == 2) {
    // no d/dz output: thread (l, u, p) takes one parity of psi into the free d/dz
    // region, then every thread sums half a line's points of both parities and stores
    const int lo = threadIdx.x & 7, u = (threadIdx.x >> 3) & 15, p = threadIdx.x >> 7;
    float2 w[16];
    const float2 *xs = X + (p * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
#pragma unroll
    for (int q = 0; q < 16; ++q) w[q] = xs[q];
    if (p) par_inv2<1>(w);
    else par_inv2<0>(w);
    float2 *xd = X + ((2 + p) * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
#pragma unroll
    for (int q = 0; q < 16; ++q) xd[q] = w[q];
    __syncthreads();
    const int hs = p;  // this thread stores s in [8 hs, 8 hs + 8)
    const float2 *y0 = X + (2 * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
    const float2 *y1 = X + (3 * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
    float2 *I2 = reinterpret_cast<float2 *>(P.I2) + slot_off + (((size_t)2 * S + kxl) * nuz) * 512 + ky0 + lo;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int sidx = 8 * hs + q;
      const int z = u + 16 * sidx;
      if (z < nuz) __stcg(&I2[(size_t)z * 512], cadd(y0[sidx], y1[sidx]));
    }
    return;
  }
  {
    // inverse stage 2: thread (l, u, o), l fastest; both parities summed; rows of I2 along k'y
    const int lo = threadIdx.x & 7, u = (threadIdx.x >> 3) & 15, o = threadIdx.x >> 7;
    {
      float2 acc[16];
      {
        const float2 *xs = X + ((2 * o) * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = xs[q];
        par_inv2<0>(acc);
      }
      {
        float2 w[16];
        const float2 *xs = X + ((2 * o + 1) * SF_PAR_ZS_ROWS + lo) * SF_PAR_LS8 + 17 * u;
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = xs[q];
        par_inv2<1>(w);
#pragma unroll
        for (int s = 0; s < 16; ++s) acc[s] = cadd(acc[s], w[s]);
      }
      const int f = o == 0 ? c : 3 + c;
      float2 *I2 = reinterpret_cast<float2 *>(P.I2) + slot_off + (((size_t)f * S + kxl) * nuz) * 512 + ky0 + lo;
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const int z = u + 16 * s;
        if (z < nuz) __stcg(&I2[(size_t)z * 512], acc[s]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// YI: 16 z rows (fixed f, kx) of I2 along k'y; the curl outputs are formed in
// y-spectral space on the way in: u_x = i ky psi_z - d/dz psi_y,
// u_y = d/dz psi_x - i kx psi_z, u_z = i (kx psi_y - ky psi_x); inverse of
// both y parities, summed -> B [f][kx][z][y]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void par_yi(const Prob<float> &P, int S, size_t slot_off, int kx0, int nkx, int tile,
                                       float2 *X) {
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, SF_PAR_YI_ROWS);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % nkx;
  const int f = rest / nkx;
  if (f >= P.nout) return;  // uniform over the block
  const int kx = kx0 + kxl;
  const int z0 = iz * SF_PAR_YI_ROWS;
  const float2 *twp = P.ax[1].twf + SF_TWP_OFF;
  // fields of I2: 0..2 psi, 3 d/dz psi_x, 4 d/dz psi_y
  const int fa = f < 3 ? f : (f == 3 ? 2 : (f == 4 ? 3 : 1));
  const int fb = f == 3 ? 4 : (f == 4 ? 2 : 0);
  {
    // inverse stage 1: thread (k1, l), k1 fastest (contiguous row loads)
    const int k1 = threadIdx.x & 15, l = threadIdx.x >> 4;
    const int z = z0 + l;
    const bool ok = z < nuz;
    const float2 *I2 = reinterpret_cast<const float2 *>(P.I2) + slot_off;
    const float2 *ra = I2 + (((size_t)fa * S + kxl) * nuz + (ok ? z : 0)) * 512 + k1;
    const float2 *rb = I2 + (((size_t)fb * S + kxl) * nuz + (ok ? z : 0)) * 512 + k1;
    const float kxv = __ldg(&P.ax[0].kap[kx]);
    const float ky1 = __ldg(&P.ax[1].kap[1]);
#pragma unroll
    for (int py = 0; py < 2; ++py) {
      float2 v[16];
      if (f < 3) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) v[k2] = ok ? __ldcg(&ra[256 * py + 16 * k2]) : czero<float2>();
      } else {
        float2 b[16];
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          v[k2] = ok ? __ldcg(&ra[256 * py + 16 * k2]) : czero<float2>();
          b[k2] = ok ? __ldcg(&rb[256 * py + 16 * k2]) : czero<float2>();
        }
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          const float kyv = par_kap(py, k1 + 16 * k2, ky1);
          if (f == 3) v[k2] = csub(mul_i(cscale(v[k2], kyv)), b[k2]);
          else if (f == 4) v[k2] = csub(v[k2], mul_i(cscale(b[k2], kxv)));
          else v[k2] = mul_i(csub(cscale(v[k2], kxv), cscale(b[k2], kyv)));
        }
      }
      if (py) par_inv1<1>(v, twp, k1);
      else par_inv1<0>(v, twp, k1);
      float2 *xd = X + (py * 16 + l) * SF_PAR_LS16 + k1;
#pragma unroll
      for (int uu = 0; uu < 16; ++uu) xd[17 * uu] = v[uu];
    }
  }
  __syncthreads();
  {
    // inverse stage 2: thread (u, l), u fastest; rows of B stored along y
    const int u = threadIdx.x & 15, l = threadIdx.x >> 4;
    float2 acc[16];
    {
      const float2 *xs = X + l * SF_PAR_LS16 + 17 * u;
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = xs[q];
      par_inv2<0>(acc);
    }
    {
      float2 w[16];
      const float2 *xs = X + (16 + l) * SF_PAR_LS16 + 17 * u;
#pragma unroll
      for (int q = 0; q < 16; ++q) w[q] = xs[q];
      par_inv2<1>(w);
#pragma unroll
      for (int s = 0; s < 16; ++s) acc[s] = cadd(acc[s], w[s]);
    }
    const int z = z0 + l;
    if (z < nuz) {
      float2 *dst = reinterpret_cast<float2 *>(P.B) + (((size_t)f * nsx + kx) * nuz + z) * nuy;
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const int y = u + 16 * s;
        if (y < nuy) __stcs(&dst[y], acc[s]);
      }
    }
  }
}

}  // namespace sfg
