// sf_fast.cuh -- register-resident fast path for periodic / unbounded 3D FP32
// solves whose three axes share one FFT length L = 32*E (E = 8 or 16, i.e.
// L = 256 or 512).
//
// Warp FFT.  One warp owns one line of L points; thread t holds x[t + 32 r],
// r < E.  The transform is the four-step split L = E x 32:
//   1. E-point DFT over r in registers, twiddle by W_L^{t k1};
//   2. one transpose through the warp's own shared buffer;
//   3. the 32-point DFTs over t as (E in registers) x (G = 32/E across lanes):
//      E-point DFT in registers, twiddle W_32^{q j}, then a radix-2
//      decimation-in-frequency network over the G lanes (warp shuffles).
// Output "k layout": lane t = (k1 = t/G, q = t%G), register j holds
// X[k1 + E (j + E bitrev_G(q))].  The inverse runs the transposed network
// (decimation in time over lanes, conjugate twiddles) from the k layout back
// to the natural layout.  Only __syncwarp is needed inside a transform.
// For the doubled (unbounded) axes the upper half of every forward input is
// zero and only the lower half of every inverse output is kept: the first /
// last E-point DFT is then evaluated in a pruned form.
//
// Pass structure (every global access is a contiguous row or a >= 64-byte
// chunk of a shared-memory transpose):
//   k_fx   source rows along x  -> A  [c][kx][z][y]     (transposed store, 16 y per chunk)
//   YF     rows of A along y    -> I1 [c][kx][ky][z]    (transposed store, 16 z per chunk)
//   ZS     rows of I1 along z: forward, multiply, operator, inverse
//                               -> I2 [f][kx][ky][z]    (direct row store), or, for the
//                                  split curl, I2 [f][kx][z][ky] (64-byte chunks)
//   YI     columns of I2 along ky (transposed load), or whole ky rows of the
//          split layout         -> B  [f][kx][z][y]     (direct row store)
//   k_fxi  B transposed back    -> result rows along x
// YF/ZS/YI run in one persistent kernel over slabs of S kx-planes; I1 and I2
// are rings of D + 2 slabs (D = stage lag) so that they stay resident in L2
// while the slab pipeline (YF of slab s, ZS of s-D, YI of s-2D) advances.
// The 3-component curl is split by component in the z stage: it emits psi_c
// and, for c = x, y, d/dz psi_c (5 z inverses per (kx, ky) instead of 6), and
// the y inverse forms u = curl psi from them in y-spectral space.
#pragma once

#include <atomic>

#include "sf_kernels.cuh"
#include "sf_par.cuh"

namespace sfg {

#define SF_FAST_THREADS 256
static_assert(SF_FAST_THREADS == SF_PAR_THREADS, "one CTA size for every fast-path tile");

// The warp FFT (wfft_fwd_m / wfft_inv_m, klayout, wrow) is defined in
// sf_device.cuh, where the general engine also uses it for L = 256 / 512.

// ---------------------------------------------------------------------------
// fast pass descriptors (YZ executor)
// ---------------------------------------------------------------------------
enum FastKind : int { FK_YF = 0, FK_ZS = 1, FK_YI = 2 };

struct FPass {
  int kind;
  int kx0, nkx;  // kx planes of the slab
  int slot;      // ring slot of I1 / I2
  int ntiles;
  int dep[2];
  int depcnt[2];
};

struct FastGeo {
  int S;      // planes per ring slot
  int nslot;  // ring slots
  int nfmax;  // fields per slot
};

#define SF_YZ_MAXM 3  // interleaved lines per warp in the YZ executor (z stage with 3 components)
// warp-buffer depth of an executor variant: the split-curl variant (OPS = 2)
// keeps one line per warp so that two CTAs fit on an SM
__host__ __device__ constexpr int fast_yz_lines(int ops) { return ops >= 2 ? 1 : SF_YZ_MAXM; }
template <int E, int M> __host__ __device__ constexpr int fast_wsm_elems() { return 8 * M * E * wrow<E>(); }

// tiles of the YZ passes (the device decoders below use the same geometry)
#define SF_YF_ROWS 16  // z rows per YF tile
#define SF_ZS_ROWS 8   // ky rows per ZS tile (one per warp)
#define SF_YI_COLS 16  // z columns per YI tile
// z rows per YI tile of the split curl: 4 per warp on 512-point axes, 2 on
// 256-point axes (whose smaller slabs would otherwise leave CTAs idle)
__host__ __device__ constexpr int fast_yi_split_rows(int L) { return L == 512 ? 32 : 16; }
template <typename T> __host__ __device__ inline int fast_tiles_yf(const Prob<T> &Q, int nkx) {
  return Q.nin * nkx * cdiv(Q.nuz, SF_YF_ROWS);
}
// forward 3D curl solved component by component (the z stage emits psi_c and
// d/dz psi_c; the x / y derivatives are applied in y-spectral space by YI)
template <typename T> __host__ __device__ inline bool fast_split_curl(const Prob<T> &Q) {
  return Q.op == OPK_CURL && Q.ncomp == 3 && Q.dim == 3 && !Q.adjoint;
}
__host__ __device__ inline int fast_tiles_zs(int nkx, int L) { return nkx * (L / SF_ZS_ROWS); }
// forward 3D curl on zero-padded 512-point axes: the parity-split y / z stages (sf_par.cuh)
template <typename T> __host__ __device__ inline bool fast_par(const Prob<T> &Q) {
  return fast_split_curl(Q) && Q.ax[0].kind == AK_U && Q.ax[0].L == 512 && Q.ax[1].L == 512 && Q.ax[2].L == 512;
}
template <typename T> __host__ __device__ inline int fast_tiles_yi(const Prob<T> &Q, int nkx) {
  const int rows = fast_par(Q) ? SF_PAR_YI_ROWS : (fast_split_curl(Q) ? fast_yi_split_rows(Q.ax[1].L) : SF_YI_COLS);
  return Q.nout * nkx * cdiv(Q.nuz, rows);
}

// Row stride (complex elements) of the 16-line transpose tile of the x
// inverse transform.  With 512 points the rows are 18 apart, so that the two
// columns of a line pair are read as one 16-byte load (k layout, 8 lanes
// per quarter warp; the only bank conflict is a 2-way one between lanes 0
// and 1); 256-point lines keep 17.  The x forward tile keeps stride 17.
template <int E> __host__ __device__ constexpr int xts() { return E == 16 ? 18 : 17; }
// the two columns (a, b) of one line pair at element i of the tile (i even
// when the stride is: one 16-byte load)
template <int TS, typename V> __device__ __forceinline__ void col_pair(const V *T, int i, V &a, V &b) {
  if constexpr (TS % 2 == 0) {
    const float4 r = *reinterpret_cast<const float4 *>(&T[i]);
    a = mk<V>(r.x, r.y);
    b = mk<V>(r.z, r.w);
  } else {
    a = T[i];
    b = T[i + 1];
  }
}

// ---------------------------------------------------------------------------
// XFWD: 16 source lines (8 packed pairs, one per warp) -> A[c][kx][z][y]
// ---------------------------------------------------------------------------
template <int E, bool PAD>
__global__ void __launch_bounds__(SF_FAST_THREADS, 5) k_fx(const Prob<float> *probs, IOArgs<float> io) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  load_prob<float>(sP, probs, io);
  const Prob<float> &P = sP;
  // one region: the warp buffers during the transform, then the output tile
  V *T = reinterpret_cast<V *>(fsm);
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  V *wsm = T + warp * E * wrow<E>();
  const Axis<float> &X = P.ax[0], &Y = P.ax[1];
  const int nuy = P.nuy, nuz = P.nuz, nux = X.nu, nsx = P.nsx;
  const int ty = cdiv(nuy, 16);
  const int tile = blockIdx.x;
  const int iy = tile % ty;
  const int rest = tile / ty;
  const int qz = rest % nuz;
  const int c = rest / nuz;
  const int y0 = iy * 16;
  const int la = y0 + 2 * warp, lb = la + 1;
  if (c >= P.nin) return;
  const float *src = P.in_ptr[c];
  V vv[1][E];
  V *v = vv[0];
  {
    const size_t rowa = ((size_t)qz * Y.nodes + la) * X.nodes;
    const size_t rowb = rowa + X.nodes;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      float a = 0.f, b = 0.f;
      if ((!PAD || r < E / 2) && src && pos < nux) {
        if (la < nuy) a = __ldcs(&src[rowa + pos]);
        if (lb < nuy) b = __ldcs(&src[rowb + pos]);
      }
      v[r] = mk<V>(a, b);
    }
  }
  wfft_fwd_m<float, E, PAD, 1>(vv, wsm, X.twf);
  // natural order in the warp buffer (one pad slot per 32) for the Hermitian split
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = klayout<E>(t, j);
    wsm[k + (k >> 5)] = v[j];
  }
  __syncwarp();
  const int half = L / 2;
  // Hermitian split into registers (k = t + 32 i <= L/2), then the tile
  // overwrites the warp buffers of all warps
  constexpr int NK = (16 * E) / 32 + 1;
  V sa[NK], sb[NK];
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int k = t + 32 * i;
    if (k <= half) {
      const int km = (L - k) & (L - 1);
      const V zk = wsm[k + (k >> 5)];
      const V zm = wsm[km + (km >> 5)];
      sa[i] = mk<V>((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
      sb[i] = mk<V>((zk.y + zm.y) * 0.5f, -(zk.x - zm.x) * 0.5f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int k = t + 32 * i;
    if (k <= half) {
      T[k * 17 + 2 * warp] = sa[i];
      T[k * 17 + 2 * warp + 1] = sb[i];
    }
  }
  __syncthreads();
  V *out = reinterpret_cast<V *>(P.A);
  const size_t plane = (size_t)nuz * nuy;
  if ((nuy & 1) == 0) {
    // pairs of y as 16-byte stores (y0 and nuy even keep every pair aligned and inside the row)
    const int cnt = (half + 1) * 8;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l2 = e & 7, kx = e >> 3;
      if (y0 + 2 * l2 < nuy) {
        const V a = T[kx * 17 + 2 * l2], b = T[kx * 17 + 2 * l2 + 1];
        float4 *dst = reinterpret_cast<float4 *>(out + ((size_t)c * nsx + kx) * plane + (size_t)qz * nuy + y0 + 2 * l2);
        *dst = make_float4(a.x, a.y, b.x, b.y);
      }
    }
  } else {
    const int cnt = (half + 1) * 16;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l = e & 15, kx = e >> 4;
      if (y0 + l < nuy) out[((size_t)c * nsx + kx) * plane + (size_t)qz * nuy + y0 + l] = T[kx * 17 + l];
    }
  }
}

// ---------------------------------------------------------------------------
// XINV: B[f][kx][z][y0..y0+16) -> 16 result lines along x
// ---------------------------------------------------------------------------
// shared memory of k_fx / k_fxi: one region that serves as the 16-line
// transpose tile and, at another time, as the warp buffers
template <int E> __host__ __device__ constexpr int fast_xi_elems() {
  return (16 * E + 1) * xts<E>() > fast_wsm_elems<E, 1>() ? (16 * E + 1) * xts<E>() : fast_wsm_elems<E, 1>();
}

template <int E, bool PAD>
__global__ void __launch_bounds__(SF_FAST_THREADS, 5) k_fxi(const Prob<float> *probs, IOArgs<float> io) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  load_prob<float>(sP, probs, io);
  const Prob<float> &P = sP;
  V *T = reinterpret_cast<V *>(fsm);
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  V *wsm = T + warp * E * wrow<E>();
  const Axis<float> &X = P.ax[0], &Y = P.ax[1];
  const int nuy = P.nuy, nuz = P.nuz, nux = X.nu, nsx = P.nsx;
  const int ty = cdiv(nuy, 16);
  const int tile = blockIdx.x;
  const int iy = tile % ty;
  const int rest = tile / ty;
  const int qz = rest % nuz;
  const int f = rest / nuz;
  const int y0 = iy * 16;
  if (f >= P.nout) return;
  const V *in = reinterpret_cast<const V *>(P.B);
  const size_t plane = (size_t)nuz * nuy;
  const int half = L / 2;
  constexpr int TS = xts<E>();
  {
    constexpr int CNT = (16 * E + 1) * 16;
    constexpr int PER = (CNT + SF_FAST_THREADS - 1) / SF_FAST_THREADS;
    V tmp[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * SF_FAST_THREADS;
      const int l = e & 15, kx = e >> 4;
      tmp[i] = (e < CNT && y0 + l < nuy) ? __ldcs(&in[((size_t)f * nsx + kx) * plane + (size_t)qz * nuy + y0 + l])
                                         : czero<V>();
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * SF_FAST_THREADS;
      if (e < CNT) T[(e >> 4) * TS + (e & 15)] = tmp[i];
    }
  }
  __syncthreads();
  V vv[1][E];
  V *v = vv[0];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = klayout<E>(t, j);
    if (k <= half) {
      V A, B;
      col_pair<TS>(T, k * TS + 2 * warp, A, B);
      if (k == 0 || k == half) {
        A.y = 0.f;
        B.y = 0.f;
      }
      v[j] = mk<V>(A.x - B.y, A.y + B.x);
    } else {
      const int kk = L - k;
      V A, B;
      col_pair<TS>(T, kk * TS + 2 * warp, A, B);
      v[j] = mk<V>(A.x + B.y, B.x - A.y);
    }
  }
  __syncthreads();  // the tile is free: it becomes the warp buffers
  wfft_inv_m<float, E, PAD, 1>(vv, wsm, X.twf);
  const int la = y0 + 2 * warp, lb = la + 1;
  float *dst = P.out_ptr[f];
  const size_t rowa = ((size_t)qz * Y.nodes + la) * X.nodes;
  const size_t rowb = rowa + X.nodes;
#pragma unroll
  for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
    const int pos = t + 32 * r;
    if (pos < nux) {
      if (la < nuy) __stcs(&dst[rowa + pos], v[r].x);
      if (lb < nuy) __stcs(&dst[rowb + pos], v[r].y);
    }
  }
}

// ---------------------------------------------------------------------------
// YZ tiles
// ---------------------------------------------------------------------------
// YF: 16 rows (consecutive z, fixed c and kx) of A along y -> I1 slot [c][kxl][ky][z]
template <int E, bool PAD, int M2>
__device__ __forceinline__ void fast_yf(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile,
                                        cx<float> *wsm, cx<float> *T) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, SF_YF_ROWS);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % ps.nkx;
  const int c = rest / ps.nkx;
  const int kx = ps.kx0 + kxl;
  const int z0 = iz * SF_YF_ROWS;
  if (c >= P.nin) return;  // tile outside the pass (uniform over the block)
  const V *A = reinterpret_cast<const V *>(P.A);
  if (M2 == 1 && PAD) {
    // one row after the other; the (half, nonzero) input of the second row is
    // loaded with the first so that both loads share one memory latency
    const int za = z0 + 2 * warp, zb = za + 1;
    const V *sa = A + (((size_t)c * nsx + kx) * nuz + za) * nuy;
    const V *sb = A + (((size_t)c * nsx + kx) * nuz + zb) * nuy;
    V v[1][E], nb[E / 2];
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const int pos = t + 32 * r;
      v[0][r] = (za < nuz && pos < nuy) ? __ldcs(&sa[pos]) : czero<V>();
      nb[r] = (zb < nuz && pos < nuy) ? __ldcs(&sb[pos]) : czero<V>();
    }
#pragma unroll
    for (int r = E / 2; r < E; ++r) v[0][r] = czero<V>();
    wfft_fwd_m<float, E, true, 1>(v, wsm, P.ax[1].twf);
#pragma unroll
    for (int j = 0; j < E; ++j) T[trow<E>(klayout<E>(t, j)) + 2 * warp] = v[0][j];
#pragma unroll
    for (int r = 0; r < E; ++r) v[0][r] = r < E / 2 ? nb[r] : czero<V>();
    wfft_fwd_m<float, E, true, 1>(v, wsm, P.ax[1].twf);
#pragma unroll
    for (int j = 0; j < E; ++j) T[trow<E>(klayout<E>(t, j)) + 2 * warp + 1] = v[0][j];
  } else
  // two rows per warp, transformed together (M2 = 2) or one after the other (M2 = 1)
#pragma unroll
  for (int h0 = 0; h0 < 2; h0 += M2) {
    V v[M2][E];
#pragma unroll
    for (int h = 0; h < M2; ++h) {
      const int z = z0 + 2 * warp + h0 + h;
      const V *src = A + (((size_t)c * nsx + kx) * nuz + z) * nuy;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int pos = t + 32 * r;
        v[h][r] = ((!PAD || r < E / 2) && z < nuz && pos < nuy) ? __ldcs(&src[pos]) : czero<V>();
      }
    }
    wfft_fwd_m<float, E, PAD, M2>(v, wsm, P.ax[1].twf);
#pragma unroll
    for (int h = 0; h < M2; ++h)
#pragma unroll
      for (int j = 0; j < E; ++j) T[trow<E>(klayout<E>(t, j)) + 2 * warp + h0 + h] = v[h][j];
  }
  __syncthreads();
  V *I1 = reinterpret_cast<V *>(P.I1) + (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const size_t base = (((size_t)c * g.S + kxl) * L) * nuz + z0;
  if ((nuz & 1) == 0) {
    // pairs of z: 16-byte stores (z0 and nuz even keep every pair aligned and inside the row)
    float4 *I1q = reinterpret_cast<float4 *>(I1 + base);
    const int cnt = L * 8;
#pragma unroll 4
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l2 = e & 7, ky = e >> 3;
      if (z0 + 2 * l2 < nuz) {
        const V a = T[trow<E>(ky) + 2 * l2], b = T[trow<E>(ky) + 2 * l2 + 1];
        __stcg(&I1q[((size_t)ky * nuz >> 1) + l2], make_float4(a.x, a.y, b.x, b.y));
      }
    }
  } else {
    const int cnt = L * 16;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l = e & 15, ky = e >> 4;
      if (z0 + l < nuz) __stcg(&I1[base + (size_t)ky * nuz + l], T[trow<E>(ky) + l]);
    }
  }
}

// multiplier of the fast path: Green's table in [kx][ky'][kz'] order (kz fastest) or eigenvalue sum

// per-warp staging row of the Green's table in the z stage (floats; >= L / 2 + 1)
#define SF_ZS_GROW 264

__device__ __forceinline__ float fast_mult(const Prob<float> &P, int kx, int ky, int kz) {
  if (P.green) {
    const int L = P.ax[2].L;
    const int kyf = min(ky, P.ax[1].L - ky);
    const int kzf = min(kz, L - kz);
    return __ldg(&P.ghat_t[((size_t)kx * P.gny + kyf) * P.gnz + kzf]);
  }
  return multiplier<float>(P, kx, ky, kz);
}

// coefficient of component c in operator output o at wavenumber (kx, ky, kz):
//   sign * i * kappa_axis   (first derivatives),  or  -|kappa|^2  (Laplacian)
__device__ __forceinline__ cx<float> op_coef(const Prob<float> &P, int o, int c, float kx, float ky, float kz, float k2) {
  const int code = P.opc[o][c];  // 0: none, +-1: +-i kappa_axis, 2: -|kappa|^2
  if (code == 0) return czero<cx<float>>();
  if (code == 2) return mk<cx<float>>(-k2, 0.f);
  const int ax = P.opa[o][c];
  const float kk = ax == 0 ? kx : (ax == 1 ? ky : kz);
  return mk<cx<float>>(0.f, code > 0 ? kk : -kk);
}

// ZS: 8 rows (consecutive ky, fixed kx) of I1 along z: forward, multiply,
// operator, inverse -> I2 rows.  Templated on the component count so that the
// spectra stay in registers; no block-wide synchronisation.
// OPS = 1: 3D curl written out (u = i kappa x psi); OPS = 0: coefficient table (any operator or none)
template <int E, int NC, bool PAD, int OPS>
__device__ __forceinline__ void fast_zs_row(const Prob<float> &P, const FastGeo &g, const FPass &ps, int kxl, int ky,
                                            cx<float> *wsm);

template <int E, int NC, bool PAD, int OPS>
__device__ __forceinline__ void fast_zs(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile,
                                        cx<float> *wsm) {
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5;
  const int nty = L / SF_ZS_ROWS;
  const int iy = tile % nty;
  const int kxl = tile / nty;
  if (kxl >= ps.nkx) return;
#pragma unroll 1
  for (int h = 0; h < SF_ZS_ROWS / 8; ++h) fast_zs_row<E, NC, PAD, OPS>(P, g, ps, kxl, iy * SF_ZS_ROWS + 8 * h + warp, wsm);
}

template <int E, int NC, bool PAD, int OPS>
__device__ __forceinline__ void fast_zs_row(const Prob<float> &P, const FastGeo &g, const FPass &ps, int kxl, int ky,
                                            cx<float> *wsm) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int t = threadIdx.x & 31;
  const int nuz = P.nuz;
  const int kx = ps.kx0 + kxl;
  const int nop = P.nop;
  const size_t slot = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *I1 = reinterpret_cast<const V *>(P.I1) + slot;
  V *I2 = reinterpret_cast<V *>(P.I2) + slot;
  const V *tz = P.ax[2].twf;
  V sp[NC][E];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const V *src = I1 + (((size_t)c * g.S + kxl) * L + ky) * nuz;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      sp[c][r] = ((!PAD || r < E / 2) && pos < nuz) ? __ldcg(&src[pos]) : czero<V>();
    }
  }
  wfft_fwd_m<float, E, PAD, NC>(sp, wsm, tz);
  const bool hasop = nop > 0;
  const float kxv = hasop ? __ldg(&P.ax[0].kap[kx]) : 0.f;
  const float kyv = hasop ? __ldg(&P.ax[1].kap[ky]) : 0.f;
  const float k2xy = hasop ? __ldg(&P.ax[0].kap2[kx]) + __ldg(&P.ax[1].kap2[ky]) : 0.f;
  if (P.adjoint) {
    for (int o = 0; o < nop; ++o) {
      V gvv[1][E];
      V *gv = gvv[0];
      const V *src = I1 + (((size_t)(NC + o) * g.S + kxl) * L + ky) * nuz;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int pos = t + 32 * r;
        gv[r] = ((!PAD || r < E / 2) && pos < nuz) ? __ldcg(&src[pos]) : czero<V>();
      }
      wfft_fwd_m<float, E, PAD, 1>(gvv, wsm, tz);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int kz = klayout<E>(t, j);
        const float kzv = __ldg(&P.ax[2].kap[kz]);
        const float k2 = k2xy + __ldg(&P.ax[2].kap2[kz]);
#pragma unroll
        for (int c = 0; c < NC; ++c)  // conjugate transpose of the operator
          sp[c][j] = cadd(sp[c][j], cmulc(gv[j], op_coef(P, o, c, kxv, kyv, kzv, k2)));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const float m = fast_mult(P, kx, ky, klayout<E>(t, j));
#pragma unroll
    for (int c = 0; c < NC; ++c) sp[c][j] = cscale(sp[c][j], m);
  }
  if (!P.adjoint) {
    for (int o = 0; o < nop; ++o) {
      V uu[1][E];
      V *u = uu[0];
      if (OPS == 1 && NC == 3) {
        // u_o = i (kappa x psi)_o with the wavenumber pair of output o
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const float kzv = __ldg(&P.ax[2].kap[klayout<E>(t, j)]);
          V d;
          if (o == 0) d = csub(cscale(sp[2 % NC][j], kyv), cscale(sp[1 % NC][j], kzv));
          else if (o == 1) d = csub(cscale(sp[0][j], kzv), cscale(sp[2 % NC][j], kxv));
          else d = csub(cscale(sp[1 % NC][j], kxv), cscale(sp[0][j], kyv));
          u[j] = mul_i(d);
        }
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int kz = klayout<E>(t, j);
          const float kzv = __ldg(&P.ax[2].kap[kz]);
          const float k2 = k2xy + __ldg(&P.ax[2].kap2[kz]);
          V acc = czero<V>();
#pragma unroll
          for (int c = 0; c < NC; ++c) acc = cadd(acc, cmul(sp[c][j], op_coef(P, o, c, kxv, kyv, kzv, k2)));
          u[j] = acc;
        }
      }
      wfft_inv_m<float, E, PAD, 1>(uu, wsm, tz);
      V *dst = I2 + (((size_t)(NC + o) * g.S + kxl) * L + ky) * nuz;
#pragma unroll
      for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
        const int z = t + 32 * r;
        if (z < nuz) __stcg(&dst[z], u[r]);
      }
    }
  }
  wfft_inv_m<float, E, PAD, NC>(sp, wsm, tz);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    V *dst = I2 + (((size_t)c * g.S + kxl) * L + ky) * nuz;
#pragma unroll
    for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
      const int z = t + 32 * r;
      if (z < nuz) __stcg(&dst[z], sp[c][r]);
    }
  }
}

// ZS, split curl: 8 rows (consecutive ky) of one component c.  Emits
// psi_c (I2 field c) and, for c = x, y, d/dz psi_c (I2 field 3 + c).  I2 of
// the split path is stored transposed, [f][kxl][z][ky], so that the y inverse
// reads whole ky rows: each warp leaves its z row in a shared staging block
// [z][8 ky] (8-byte slots, ky index XOR-swizzled with (z >> 1) & 7 so that
// neither the row writes nor the block reads conflict), and after one CTA
// barrier the block leaves as 64-byte [z][ky0 .. ky0 + 7] segments.
__device__ __forceinline__ int zs_stage_idx(int z, int kyl) { return z * SF_ZS_ROWS + (kyl ^ ((z >> 1) & 7)); }

template <int E, bool PAD>
__device__ __forceinline__ void fast_zs_split(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile,
                                              cx<float> *wsm, cx<float> *T) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuz = P.nuz;
  const int nty = L / SF_ZS_ROWS;
  const int iy = tile % nty;
  const int rest = tile / nty;
  const int kxl = rest % ps.nkx;
  const int c = rest / ps.nkx;
  if (c >= 3) return;  // uniform over the CTA
  const int kx = ps.kx0 + kxl;
  const int ky0 = iy * SF_ZS_ROWS;
  const int ky = ky0 + warp;
  const size_t slot = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *I1 = reinterpret_cast<const V *>(P.I1) + slot;
  V *I2 = reinterpret_cast<V *>(P.I2) + slot;
  const V *tz = P.ax[2].twf;
  // T: Green's rows (8 x SF_ZS_GROW floats, unbounded axes), then the psi and
  // d/dz staging blocks of nuz x 8 slots each (nuz = L / 2 padded, L periodic)
  static_assert(SF_ZS_ROWS == 8, "staging block is [z][8 ky]");
  static_assert(2 * SF_ZS_ROWS * 32 * E <= trows_elems<E>(), "staging blocks exceed the tile buffer");
  static_assert(SF_ZS_ROWS * SF_ZS_GROW / 2 + 2 * SF_ZS_ROWS * 16 * E <= trows_elems<E>(),
                "Green's rows and staging blocks exceed the tile buffer");
  float *gs = reinterpret_cast<float *>(T) + warp * SF_ZS_GROW;
  V *st_psi = T + (PAD ? SF_ZS_ROWS * SF_ZS_GROW / 2 : 0);
  V *st_dz = st_psi + SF_ZS_ROWS * nuz;
  // Green's row of (kx, |ky|) staged in shared memory by asynchronous copies
  // that complete while the forward transform runs (unbounded axes only)
  if (PAD && P.green) {
    const int kyf = min(ky, L - ky);
    const float *grow = P.ghat_t + ((size_t)kx * P.gny + kyf) * P.gnz;
    for (int i = t; i < P.gnz; i += 32) cp_async4(gs + i, grow + i);
    cp_async_commit();
  }
  V sp[1][E];
  {
    const V *src = I1 + (((size_t)c * g.S + kxl) * L + ky) * nuz;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      sp[0][r] = ((!PAD || r < E / 2) && pos < nuz) ? __ldcg(&src[pos]) : czero<V>();
    }
  }
  wfft_fwd_m<float, E, PAD, 1>(sp, wsm, tz);
  if (PAD && P.green) {
    cp_async_wait_all();
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int kz = klayout<E>(t, j);
      sp[0][j] = cscale(sp[0][j], gs[min(kz, L - kz)]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) sp[0][j] = cscale(sp[0][j], fast_mult(P, kx, ky, klayout<E>(t, j)));
  }
  if (c < 2) {
    const float kz1 = __ldg(&P.ax[2].kap[1]);
    V dz[1][E];
#pragma unroll
    for (int j = 0; j < E; ++j) dz[0][j] = mul_i(cscale(sp[0][j], kap_of<L>(klayout<E>(t, j), kz1)));
    wfft_inv_m<float, E, PAD, 1>(dz, wsm, tz);
#pragma unroll
    for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
      const int z = t + 32 * r;
      if (z < nuz) st_dz[zs_stage_idx(z, warp)] = dz[0][r];
    }
  }
  wfft_inv_m<float, E, PAD, 1>(sp, wsm, tz);
#pragma unroll
  for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
    const int z = t + 32 * r;
    if (z < nuz) st_psi[zs_stage_idx(z, warp)] = sp[0][r];
  }
  __syncthreads();
  const int nel = nuz * SF_ZS_ROWS;
  V *dpsi = I2 + (((size_t)c * g.S + kxl) * nuz) * L + ky0;
  V *ddz = I2 + (((size_t)(3 + c) * g.S + kxl) * nuz) * L + ky0;
  for (int e = threadIdx.x; e < nel; e += SF_FAST_THREADS) {
    const int z = e >> 3, kyl = e & 7;
    const int si = zs_stage_idx(z, kyl);
    __stcg(&dpsi[(size_t)z * L + kyl], st_psi[si]);
    if (c < 2) __stcg(&ddz[(size_t)z * L + kyl], st_dz[si]);
  }
}

// YI of the split path: whole ky rows of the transposed I2 [f][kxl][z][ky],
// loaded directly in the k layout of the inverse transform (for every
// register j the 32 lanes cover two runs of 16 consecutive ky), the curl
// outputs combined in y-spectral space on the way in; fast_yi_split_rows(L) / 8 z rows per warp.
template <int E, bool PAD>
__device__ __forceinline__ void fast_yi_rows(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile,
                                             cx<float> *wsm) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  constexpr int ROWS = fast_yi_split_rows(L);
  constexpr int RPW = ROWS / (SF_FAST_THREADS / 32);  // rows per warp
  static_assert(RPW >= 1 && RPW * (SF_FAST_THREADS / 32) == ROWS, "rows per YI tile");
  const int tz = cdiv(nuz, ROWS);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % ps.nkx;
  const int f = rest / ps.nkx;
  const int kx = ps.kx0 + kxl;
  if (f >= P.nout) return;
  const size_t slot = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *I2 = reinterpret_cast<const V *>(P.I2) + slot;
  // u_x = i ky psi_z - dz psi_y, u_y = dz psi_x - i kx psi_z, u_z = i kx psi_y - i ky psi_x
  // (fields 0..2 psi, 3 dz psi_x, 4 dz psi_y)
  const int fa = f < 3 ? f : (f == 3 ? 2 : (f == 4 ? 3 : 1));
  const int fb = f == 3 ? 4 : (f == 4 ? 2 : 0);
  const float kxv = __ldg(&P.ax[0].kap[kx]);
  const float ky1 = __ldg(&P.ax[1].kap[1]);
#pragma unroll 1
  for (int h = 0; h < RPW; ++h) {
    const int z = iz * ROWS + RPW * warp + h;
    if (z >= nuz) break;  // uniform over the warp
    const V *ra = I2 + (((size_t)fa * g.S + kxl) * nuz + z) * L;
    const V *rb = I2 + (((size_t)fb * g.S + kxl) * nuz + z) * L;
    V v[1][E];
    if (f < 3) {
#pragma unroll
      for (int j = 0; j < E; ++j) v[0][j] = __ldcg(&ra[klayout<E>(t, j)]);
    } else {
      V tb[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int k = klayout<E>(t, j);
        v[0][j] = __ldcg(&ra[k]);
        tb[j] = __ldcg(&rb[k]);
      }
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const float kyv = kap_of<L>(klayout<E>(t, j), ky1);
        if (f == 3) v[0][j] = csub(mul_i(cscale(v[0][j], kyv)), tb[j]);
        else if (f == 4) v[0][j] = csub(v[0][j], mul_i(cscale(tb[j], kxv)));
        else v[0][j] = mul_i(csub(cscale(v[0][j], kxv), cscale(tb[j], kyv)));
      }
    }
    wfft_inv_m<float, E, PAD, 1>(v, wsm, P.ax[1].twf);
    V *dst = reinterpret_cast<V *>(P.B) + (((size_t)f * nsx + kx) * nuz + z) * nuy;
#pragma unroll
    for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
      const int y = t + 32 * r;
      if (y < nuy) __stcs(&dst[y], v[0][r]);
    }
  }
}

// YI: 16 z-columns (fixed f and kx) of I2 [f][kxl][ky][z], transposed through
// shared memory, inverse y transform per column -> B rows along y
template <int E, bool PAD>
__device__ __forceinline__ void fast_yi(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile,
                                        cx<float> *wsm, cx<float> *T) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, SF_YI_COLS);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % ps.nkx;
  const int f = rest / ps.nkx;
  const int kx = ps.kx0 + kxl;
  const int z0 = iz * SF_YI_COLS;
  if (f >= P.nout) return;
  const size_t slot = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *I2 = reinterpret_cast<const V *>(P.I2) + slot;
  auto field = [&](int ff) { return I2 + (((size_t)ff * g.S + kxl) * L) * nuz + z0; };
  constexpr int PER = L * 16 / SF_FAST_THREADS;
  const V *src = field(f);
  // all loads of the tile in flight before the first shared store
  V tmp[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * SF_FAST_THREADS;
    const int l = e & 15, ky = e >> 4;
    tmp[i] = (z0 + l < nuz) ? __ldcg(&src[(size_t)ky * nuz + l]) : czero<V>();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * SF_FAST_THREADS;
    T[trow<E>(e >> 4) + (e & 15)] = tmp[i];
  }
  __syncthreads();
  {
    V v[2][E];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < E; ++j) v[h][j] = T[trow<E>(klayout<E>(t, j)) + 2 * warp + h];
    wfft_inv_m<float, E, PAD, 2>(v, wsm, P.ax[1].twf);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int z = z0 + 2 * warp + h;
      if (z < nuz) {
        V *dst = reinterpret_cast<V *>(P.B) + (((size_t)f * nsx + kx) * nuz + z) * nuy;
#pragma unroll
        for (int r = 0; r < (PAD ? E / 2 : E); ++r) {
          const int y = t + 32 * r;
          if (y < nuy) __stcs(&dst[y], v[h][r]);
        }
      }
    }
  }
}

// persistent YZ executor over the slab work list (same queue / bounded-wait
// protocol as k_exec).  The pass table is packed into shared memory at start.
// Thread 0 prepares the next item during the current tile: at the start of
// tile k it decodes item k + 1 (claimed one tile earlier) and issues the loads
// of that item's dependency counters, whose L2 round trip then overlaps the
// tile; at the end of tile k it checks the loaded counts, without blocking
// (item k + 1 may depend on the very tile this CTA is still finishing), and
// claims the item after it.  The end-of-tile barrier then both completes tile
// k and publishes the prepared descriptor, so an item whose dependencies were
// met at the probe starts without a second barrier; otherwise thread 0 waits
// (bounded) while the CTA holds at one extra barrier.  Thread 32 publishes
// the completed tile with a release reduction after the barrier.  The
// descriptor is double-buffered: slot k & 1 is read during tile k while slot
// (k + 1) & 1 is written.
// OPS: 0 any operator (coefficient table), 1 curl written out, 2 split curl,
// 3 split curl with the parity-split y / z stages (zero-padded 512-point axes)
template <int E, int OPS> __host__ __device__ constexpr size_t fast_yz_region() {
  return OPS == 3 ? par_smem_bytes() : (size_t)(fast_wsm_elems<E, fast_yz_lines(OPS)>() + trows_elems<E>()) * sizeof(float2);
}

template <int E, int NC, bool PAD, int OPS>
__global__ void __launch_bounds__(SF_FAST_THREADS, OPS >= 2 ? 2 : 1)
    k_fyz(const Prob<float> *probs, FastGeo g, const FPass *passes, const int *pass_start, int npass, unsigned *done,
          ExecCtl *ctl, unsigned *sticky, unsigned long long timeout_ns, IOArgs<float> io) {
  typedef cx<float> V;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  __shared__ FPass sPass[2];
  __shared__ int s_item[2], s_pass[2], s_ok[2], s_ready[2];
  load_prob<float>(sP, probs, io);
  constexpr int MM = fast_yz_lines(OPS);  // interleaved lines per warp (warp buffer depth)
  V *wsm_all = reinterpret_cast<V *>(fsm);
  V *T = wsm_all + fast_wsm_elems<E, MM>();
  V *wsm = wsm_all + (threadIdx.x >> 5) * MM * E * wrow<E>();
  // packed pass table after the tile buffer: start[npass + 1], then per pass
  // a = kind | slot << 2 | nkx << 6 | kx0 << 16 and b = (dep0 + 1) | (dep1 + 1) << 16
  int *s_start = reinterpret_cast<int *>(fsm + fast_yz_region<E, OPS>());
  int *s_pa = s_start + npass + 1;
  int *s_pb = s_pa + npass;
  for (int i = threadIdx.x; i <= npass; i += blockDim.x) s_start[i] = pass_start[i];
  for (int i = threadIdx.x; i < npass; i += blockDim.x) {
    const FPass &q = passes[i];
    s_pa[i] = q.kind | (q.slot << 2) | (q.nkx << 6) | (q.kx0 << 16);
    s_pb[i] = (q.dep[0] + 1) | ((q.dep[1] + 1) << 16);
  }
  __syncthreads();
  const int total = s_start[npass];
  int next_it = 0;  // thread 0: item claimed one tile ahead (the queue round trip overlaps a tile)
  int cur = 0;      // thread 0: pass of the last item (items arrive in increasing order)

  // thread 0: decode the claimed item into slot k and issue the loads of its
  // dependency counters (early: at the start of the current tile, so that
  // their L2 round trip overlaps the tile); the values are checked by
  // finish_claim at the end of the tile, which then claims the item after it
  unsigned probe[2] = {0u, 0u}, need[2] = {0u, 0u};
  auto decode_issue = [&](int k) {
    const int it = next_it;
    s_item[k] = it;
    s_ok[k] = 1;
    s_ready[k] = 1;
    probe[0] = probe[1] = need[0] = need[1] = 0u;
    if (it >= total) return;
    while (s_start[cur + 1] <= it) ++cur;
    const int lo = cur;
    FPass &sp = sPass[k];
    const int a = s_pa[lo], b = s_pb[lo];
    sp.kind = a & 3;
    sp.slot = (a >> 2) & 15;
    sp.nkx = (a >> 6) & 1023;
    sp.kx0 = a >> 16;
    sp.ntiles = s_start[lo + 1] - s_start[lo];
    sp.dep[0] = (b & 0xffff) - 1;
    sp.dep[1] = ((b >> 16) & 0xffff) - 1;
    s_pass[k] = lo;
    for (int d = 0; d < 2; ++d) {
      const int dp = sp.dep[d];
      if (dp >= 0) {
        need[d] = (unsigned)(s_start[dp + 1] - s_start[dp]);
        probe[d] = ld_acquire(&done[dp]);
      }
    }
  };
  auto finish_claim = [&](int k) {
    if (s_item[k] >= total) return;
    const bool ready = probe[0] >= need[0] && probe[1] >= need[1];
    s_ready[k] = ready ? 1 : 0;  // ready at the first probe: no time is spent waiting
    next_it = (int)atomicAdd(&ctl->next, 1u);
  };
  // thread 0: bounded wait for the dependencies of the item in slot k (the
  // CTA stalls from here on: the time is recorded as waiting)
  auto wait_deps = [&](int k) {
    const FPass &sp = sPass[k];
    const unsigned long long tw0 = global_ns();
    for (int d = 0; d < 2; ++d) {
      const int dp = sp.dep[d];
      if (dp < 0) continue;
      const unsigned need = (unsigned)(s_start[dp + 1] - s_start[dp]);
      unsigned iters = 0;
      while (ld_acquire(&done[dp]) < need) {
        __nanosleep(64);
        if (((++iters) & 255u) == 0 && (global_ns() - tw0 > timeout_ns || iters > (1u << 28))) {
          atomicCAS(&ctl->error, 0u, 6u);
          atomicExch(&ctl->err_pass, (unsigned)s_pass[k]);
          atomicOr(sticky, 1u);
          s_ok[k] = 0;
          return;
        }
      }
    }
    atomicAdd(&ctl->wait_ns[sp.kind], global_ns() - tw0);
  };

  if (threadIdx.x == 0) {
    next_it = (int)atomicAdd(&ctl->next, 1u);
    decode_issue(0);
    finish_claim(0);
  }
  __syncthreads();
  for (int k = 0;; k ^= 1) {
    const int it = s_item[k];
    if (it >= total) break;
    // read before the slot can be rewritten (decode_issue(k) runs at the next tile's start)
    const int my_pass = s_pass[k];
    const int my_kind = sPass[k].kind;
    if (!s_ready[k]) {  // uniform over the CTA
      if (threadIdx.x == 0) wait_deps(k);
      __syncthreads();
    }
    if (threadIdx.x == 0) decode_issue(k ^ 1);  // the item after this one (claimed one tile ago)
    unsigned long long t_start = 0;  // thread 32: start of the tile (tracing)
    if (threadIdx.x == 32) t_start = global_ns();
    if (s_ok[k]) {
      const FPass &ps = sPass[k];
      const int tile = it - s_start[my_pass];
      if constexpr (OPS == 3) {
        const size_t slot_off = (size_t)ps.slot * g.nfmax * g.S * 512 * sP.nuz;
        float2 *X = reinterpret_cast<float2 *>(fsm);
        if (my_kind == FK_YF) par_yf(sP, g.S, slot_off, ps.kx0, ps.nkx, tile, X);
        else if (my_kind == FK_ZS) par_zs(sP, g.S, slot_off, ps.kx0, ps.nkx, tile, X);
        else par_yi(sP, g.S, slot_off, ps.kx0, ps.nkx, tile, X);
      } else {
        if (my_kind == FK_YF) fast_yf<E, PAD, MM == 1 ? 1 : 2>(sP, g, ps, tile, wsm, T);
        else if (my_kind == FK_ZS) {
          if (OPS == 2) fast_zs_split<E, PAD>(sP, g, ps, tile, wsm, T);
          else fast_zs<E, NC, PAD, OPS>(sP, g, ps, tile, wsm);
        } else if (OPS == 2) fast_yi_rows<E, PAD>(sP, g, ps, tile, wsm);
        else fast_yi<E, PAD>(sP, g, ps, tile, wsm, T);
      }
    }
    if (threadIdx.x == 0) finish_claim(k ^ 1);
    __syncthreads();
    if (threadIdx.x == 32) {
      red_release_add(&done[my_pass], 1u);  // publishes the tile (cumulative over the barrier above)
      atomicAdd(&ctl->busy_ns[my_kind], global_ns() - t_start);
      atomicAdd(&ctl->tiles[my_kind], 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// host side: launch of the three fast-path kernels (one instantiation per E)
// ---------------------------------------------------------------------------
struct FastLaunch {
  const Prob<float> *d_prob;
  const Prob<float> *h_prob;
  FastGeo geo;
  const FPass *d_passes;
  const int *d_start;
  unsigned *d_done;
  int npass, total;
  ExecCtl *ctl;
  unsigned *sticky;
  unsigned long long timeout_ns;
  bool front, back;
  cudaStream_t stream;
  cudaEvent_t *marks;  // 4 events around k_fx, k_fyz, k_fxi of a full solve, or nullptr
};

// defined in sf_fast8.cu / sf_fast16.cu; return a cudaError_t value
int sf_fast_launch_e8(const FastLaunch &fl, const IOArgs<float> &io, int *launches);
int sf_fast_launch_e16(const FastLaunch &fl, const IOArgs<float> &io, int *launches);

template <int E> size_t fast_x_smem() { return (size_t)fast_xi_elems<E>() * sizeof(float2); }
#define SF_FAST_MAXPASS 1024
// dynamic shared memory of k_fyz: warp buffers, tile buffer, packed pass table
template <int E, int OPS> size_t fast_yz_smem(int npass) {
  return fast_yz_region<E, OPS>() + (size_t)(3 * npass + 1) * sizeof(int);
}

template <int E, int NC, bool PAD, int OPS> int fast_launch_yz(const FastLaunch &fl, const IOArgs<float> &io) {
  static std::atomic<unsigned long long> attr{0};  // devices whose attributes are set
  if (fl.npass > SF_FAST_MAXPASS) return (int)cudaErrorInvalidValue;
  const size_t smyz = fast_yz_smem<E, OPS>(fl.npass);
  cudaError_t e;
  int adev = 0;
  if ((e = cudaGetDevice(&adev)) != cudaSuccess) return (int)e;
  const unsigned long long abit = adev < 64 ? 1ull << adev : 0ull;
  if (!abit || !(attr.load() & abit)) {
    e = cudaFuncSetAttribute(k_fyz<E, NC, PAD, OPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fast_yz_smem<E, OPS>(SF_FAST_MAXPASS));
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_fyz<E, NC, PAD, OPS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr.fetch_or(abit);
  }
  int dev = 0, nsm = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fyz<E, NC, PAD, OPS>, SF_FAST_THREADS, smyz)) != cudaSuccess)
    return (int)e;
  if (per < 1) return (int)cudaErrorLaunchOutOfResources;
  const int grid = fl.total < nsm * per ? fl.total : nsm * per;
  k_fyz<E, NC, PAD, OPS><<<grid, SF_FAST_THREADS, smyz, fl.stream>>>(fl.d_prob, fl.geo, fl.d_passes, fl.d_start, fl.npass,
                                                              fl.d_done, fl.ctl, fl.sticky, fl.timeout_ns, io);
  return (int)cudaGetLastError();
}

template <int E, bool PAD> int fast_launch_all(const FastLaunch &fl, const IOArgs<float> &io, int *launches) {
  const Prob<float> &Q = *fl.h_prob;
  const size_t smx = fast_x_smem<E>(), smxi = smx;
  static std::atomic<unsigned long long> attr{0};  // devices whose attributes are set
  cudaError_t e;
  int adev = 0;
  if ((e = cudaGetDevice(&adev)) != cudaSuccess) return (int)e;
  const unsigned long long abit = adev < 64 ? 1ull << adev : 0ull;
  if (!abit || !(attr.load() & abit)) {
    if ((e = cudaFuncSetAttribute(k_fx<E, PAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) != cudaSuccess)
      return (int)e;
    if ((e = cudaFuncSetAttribute(k_fxi<E, PAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smxi)) != cudaSuccess)
      return (int)e;
    if ((e = cudaFuncSetAttribute(k_fx<E, PAD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
      return (int)e;
    if ((e = cudaFuncSetAttribute(k_fxi<E, PAD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
      return (int)e;
    attr.fetch_or(abit);
  }
  cudaEvent_t *mk = fl.front && fl.back ? fl.marks : nullptr;
  if (mk && (e = cudaEventRecord(mk[0], fl.stream)) != cudaSuccess) return (int)e;
  if (fl.front) {
    k_fx<E, PAD><<<Q.nin * Q.nuz * cdiv(Q.nuy, 16), SF_FAST_THREADS, smx, fl.stream>>>(fl.d_prob, io);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    if ((e = cudaMemsetAsync(fl.d_done, 0, fl.npass * sizeof(unsigned), fl.stream)) != cudaSuccess) return (int)e;
    if ((e = cudaMemsetAsync(fl.ctl, 0, sizeof(ExecCtl), fl.stream)) != cudaSuccess) return (int)e;
    if (mk && (e = cudaEventRecord(mk[1], fl.stream)) != cudaSuccess) return (int)e;
    int r;
    if (E == 16 && PAD && fast_par(Q)) r = fast_launch_yz<E, 3, PAD, 3>(fl, io);
    else if (fast_split_curl(Q)) r = fast_launch_yz<E, 3, PAD, 2>(fl, io);
    else if (Q.ncomp == 3 && Q.op == OPK_CURL) r = fast_launch_yz<E, 3, PAD, 1>(fl, io);
    else if (Q.ncomp == 3) r = fast_launch_yz<E, 3, PAD, 0>(fl, io);
    else if (Q.ncomp == 2) r = fast_launch_yz<E, 2, PAD, 0>(fl, io);
    else r = fast_launch_yz<E, 1, PAD, 0>(fl, io);
    if (r) return r;
    if (mk && (e = cudaEventRecord(mk[2], fl.stream)) != cudaSuccess) return (int)e;
    if (launches) *launches += 2;
  }
  if (fl.back) {
    k_fxi<E, PAD><<<Q.nout * Q.nuz * cdiv(Q.nuy, 16), SF_FAST_THREADS, smxi, fl.stream>>>(fl.d_prob, io);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    if (mk && (e = cudaEventRecord(mk[3], fl.stream)) != cudaSuccess) return (int)e;
    if (launches) *launches += 1;
  }
  return 0;
}

}  // namespace sfg
