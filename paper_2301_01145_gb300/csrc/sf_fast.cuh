// sf_fast.cuh -- register-resident fast path for periodic / unbounded 3D solves
// whose three axes share one FFT length L = 32*E (E = 8 or 16, i.e. L = 256 or 512).
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
//
// Pass structure (all global accesses are contiguous rows or >= 64-byte
// chunks of a shared-memory transpose):
//   k_fx   source rows along x  -> A  [c][kx][z][y]      (16 y per chunk)
//   YF     rows of A along y    -> I1 [c][kx][ky][z]     (16 z per chunk)
//   ZS     rows of I1 along z: forward, multiply, operator, inverse
//                               -> I2 [f][kx][z][ky]     (8 ky per chunk)
//   YI     rows of I2 along ky  -> B  [f][kx][z][y]      (contiguous rows)
//   k_fxi  B transposed back    -> result rows along x
// YF/ZS/YI run in one persistent kernel over slabs of S kx-planes; I1 and I2
// are rings of two slabs so that they stay resident in L2 while the slab
// pipeline (YF of slab s, ZS of s-1, YI of s-2) advances.
#pragma once

#include "sf_kernels.cuh"

namespace sfg {

#define SF_FAST_THREADS 256

__device__ __forceinline__ int bitrev_lanes(int q, int G) {
  int r = 0;
  for (int b = 1; b < G; b <<= 1) {
    r = (r << 1) | (q & 1);
    q >>= 1;
  }
  return r;
}

template <typename V> __device__ __forceinline__ V shfl_xor_c(V v, int m) {
  V r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

// k index held in register j by this lane after a forward warp FFT
template <int E> __device__ __forceinline__ int klayout(int lane, int j) {
  constexpr int G = 32 / E;
  const int k1 = lane / G, q = lane % G;
  return k1 + E * (j + E * bitrev_lanes(q, G));
}

template <typename T, int E>
__device__ __forceinline__ void wfft_fwd(cx<T> *v, cx<T> *wsm, const cx<T> *__restrict__ tw) {
  typedef cx<T> V;
  constexpr int L = 32 * E, G = 32 / E;
  const int t = threadIdx.x & 31;
  dftR<E, false>(v);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], __ldg(&tw[t * k1]));
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) wsm[k1 * 33 + t] = v[k1];
  __syncwarp();
  const int k1 = t / G, q = t % G;
#pragma unroll
  for (int s = 0; s < E; ++s) v[s] = wsm[k1 * 33 + G * s + q];
  __syncwarp();
  dftR<E, false>(v);
#pragma unroll
  for (int j = 1; j < E; ++j) v[j] = cmul(v[j], __ldg(&tw[q * j * E]));
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) {
    const V w = __ldg(&tw[(q & (m - 1)) * (L / (2 * m))]);
    const bool hi = (q & m) != 0;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const V p = shfl_xor_c(v[j], m);
      v[j] = hi ? cmul(csub(p, v[j]), w) : cadd(v[j], p);
    }
  }
}

template <typename T, int E>
__device__ __forceinline__ void wfft_inv(cx<T> *v, cx<T> *wsm, const cx<T> *__restrict__ tw) {
  typedef cx<T> V;
  constexpr int L = 32 * E, G = 32 / E;
  const int t = threadIdx.x & 31;
  const int k1 = t / G, q = t % G;
#pragma unroll
  for (int m = 1; m < G; m <<= 1) {
    const V w = __ldg(&tw[(q & (m - 1)) * (L / (2 * m))]);
    const bool hi = (q & m) != 0;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const V p = shfl_xor_c(v[j], m);
      v[j] = hi ? csub(p, cmulc(v[j], w)) : cadd(v[j], cmulc(p, w));
    }
  }
#pragma unroll
  for (int j = 1; j < E; ++j) v[j] = cmulc(v[j], __ldg(&tw[q * j * E]));
  dftR<E, true>(v);
#pragma unroll
  for (int s = 0; s < E; ++s) wsm[k1 * 33 + G * s + q] = v[s];
  __syncwarp();
#pragma unroll
  for (int kk = 0; kk < E; ++kk) v[kk] = wsm[kk * 33 + t];
  __syncwarp();
#pragma unroll
  for (int kk = 1; kk < E; ++kk) v[kk] = cmulc(v[kk], __ldg(&tw[t * kk]));
  dftR<E, true>(v);
}

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
  int S;        // planes per ring slot
  int nslot;    // ring slots
  int nfmax;    // fields per slot
};

template <int E> __host__ __device__ constexpr int fast_wsm_elems() { return 8 * E * 33; }

// ---------------------------------------------------------------------------
// XFWD: 16 source lines (8 packed pairs, one per warp) -> A[c][kx][z][y]
// ---------------------------------------------------------------------------
template <int E>
__global__ void __launch_bounds__(SF_FAST_THREADS) k_fx(const Prob<float> *probs, IOArgs<float> io) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  load_prob<float>(sP, probs, io);
  const Prob<float> &P = sP;
  V *wsm_all = reinterpret_cast<V *>(fsm);
  V *T = wsm_all + fast_wsm_elems<E>();
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  V *wsm = wsm_all + warp * E * 33;
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
  const float *src = P.in_ptr[c];
  V v[E];
  {
    const size_t rowa = ((size_t)qz * Y.nodes + la) * X.nodes;
    const size_t rowb = rowa + X.nodes;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      float a = 0.f, b = 0.f;
      if (src && pos < nux) {
        if (la < nuy) a = __ldcs(&src[rowa + pos]);
        if (lb < nuy) b = __ldcs(&src[rowb + pos]);
      }
      v[r] = mk<V>(a, b);
    }
  }
  wfft_fwd<float, E>(v, wsm, X.tw);
  // natural order in the warp buffer (one pad slot per 32) for the Hermitian split
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = klayout<E>(t, j);
    wsm[k + (k >> 5)] = v[j];
  }
  __syncwarp();
  const int half = L / 2;
  for (int k = t; k <= half; k += 32) {
    const int km = (L - k) & (L - 1);
    const V zk = wsm[k + (k >> 5)];
    const V zm = wsm[km + (km >> 5)];
    T[k * 17 + 2 * warp] = mk<V>((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
    T[k * 17 + 2 * warp + 1] = mk<V>((zk.y + zm.y) * 0.5f, -(zk.x - zm.x) * 0.5f);
  }
  __syncthreads();
  V *out = reinterpret_cast<V *>(P.A);
  const size_t plane = (size_t)nuz * nuy;
  const int cnt = (half + 1) * 16;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int l = e & 15, kx = e >> 4;
    if (y0 + l < nuy) out[((size_t)c * nsx + kx) * plane + (size_t)qz * nuy + y0 + l] = T[kx * 17 + l];
  }
}

// ---------------------------------------------------------------------------
// XINV: B[f][kx][z][y0..y0+16) -> 16 result lines along x
// ---------------------------------------------------------------------------
template <int E>
__global__ void __launch_bounds__(SF_FAST_THREADS) k_fxi(const Prob<float> *probs, IOArgs<float> io) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  load_prob<float>(sP, probs, io);
  const Prob<float> &P = sP;
  V *wsm_all = reinterpret_cast<V *>(fsm);
  V *T = wsm_all + fast_wsm_elems<E>();
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  V *wsm = wsm_all + warp * E * 33;
  const Axis<float> &X = P.ax[0], &Y = P.ax[1];
  const int nuy = P.nuy, nuz = P.nuz, nux = X.nu, nsx = P.nsx;
  const int ty = cdiv(nuy, 16);
  const int tile = blockIdx.x;
  const int iy = tile % ty;
  const int rest = tile / ty;
  const int qz = rest % nuz;
  const int f = rest / nuz;
  const int y0 = iy * 16;
  const V *in = reinterpret_cast<const V *>(P.B);
  const size_t plane = (size_t)nuz * nuy;
  const int half = L / 2;
  const int cnt = (half + 1) * 16;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int l = e & 15, kx = e >> 4;
    T[kx * 17 + l] = (y0 + l < nuy) ? __ldcs(&in[((size_t)f * nsx + kx) * plane + (size_t)qz * nuy + y0 + l])
                                    : czero<V>();
  }
  __syncthreads();
  V v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = klayout<E>(t, j);
    if (k <= half) {
      V A = T[k * 17 + 2 * warp], B = T[k * 17 + 2 * warp + 1];
      if (k == 0 || k == half) {
        A.y = 0.f;
        B.y = 0.f;
      }
      v[j] = mk<V>(A.x - B.y, A.y + B.x);
    } else {
      const int kk = L - k;
      const V A = T[kk * 17 + 2 * warp], B = T[kk * 17 + 2 * warp + 1];
      v[j] = mk<V>(A.x + B.y, B.x - A.y);
    }
  }
  wfft_inv<float, E>(v, wsm, X.tw);
  const int la = y0 + 2 * warp, lb = la + 1;
  float *dst = P.out_ptr[f];
  const size_t rowa = ((size_t)qz * Y.nodes + la) * X.nodes;
  const size_t rowb = rowa + X.nodes;
#pragma unroll
  for (int r = 0; r < E; ++r) {
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
template <int E>
__device__ void fast_yf(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile, cx<float> *wsm, cx<float> *T) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, 16);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % ps.nkx;
  const int c = rest / ps.nkx;
  const int kx = ps.kx0 + kxl;
  const int z0 = iz * 16;
  const V *A = reinterpret_cast<const V *>(P.A);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int row = 2 * warp + h;
    const int z = z0 + row;
    V v[E];
    const V *src = A + (((size_t)c * nsx + kx) * nuz + z) * nuy;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      v[r] = (z < nuz && pos < nuy) ? __ldcs(&src[pos]) : czero<V>();
    }
    wfft_fwd<float, E>(v, wsm, P.ax[1].tw);
#pragma unroll
    for (int j = 0; j < E; ++j) T[klayout<E>(t, j) * 17 + row] = v[j];
  }
  __syncthreads();
  V *I1 = reinterpret_cast<V *>(P.I1) + (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const size_t base = (((size_t)c * g.S + kxl) * L) * nuz + z0;
  const int cnt = L * 16;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int l = e & 15, ky = e >> 4;
    if (z0 + l < nuz) __stcg(&I1[base + (size_t)ky * nuz + l], T[ky * 17 + l]);
  }
}

// ZS: 8 rows (consecutive ky, fixed kx) of I1 along z: forward, multiply, operator, inverse -> I2 slot
template <int E>
__device__ void fast_zs(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile, cx<float> *wsm, cx<float> *T) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuz = P.nuz;
  const int nty = L / 8;
  const int iy = tile % nty;
  const int kxl = tile / nty;
  const int kx = ps.kx0 + kxl;
  const int ky0 = iy * 8;
  const int ky = ky0 + warp;
  const int ncomp = P.ncomp, nop = P.nop;
  const size_t slotI1 = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *I1 = reinterpret_cast<const V *>(P.I1) + slotI1;
  V *I2 = reinterpret_cast<V *>(P.I2) + slotI1;
  const Axis<float> &Z = P.ax[2];
  auto load_fwd = [&](int field, V *v) {
    const V *src = I1 + (((size_t)field * g.S + kxl) * L + ky) * nuz;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int pos = t + 32 * r;
      v[r] = pos < nuz ? __ldcg(&src[pos]) : czero<V>();
    }
    wfft_fwd<float, E>(v, wsm, Z.tw);
  };
  auto inv_store = [&](int field, V *v) {
    wfft_inv<float, E>(v, wsm, Z.tw);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int z = t + 32 * r;
      if (z < nuz) T[z * 9 + warp] = v[r];
    }
    __syncthreads();
    V *dst = I2 + (((size_t)field * g.S + kxl) * nuz) * L + ky0;
    const int cnt = nuz * 8;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l = e & 7, z = e >> 3;
      __stcg(&dst[(size_t)z * L + l], T[z * 9 + l]);
    }
    __syncthreads();
  };
  V ps_[3][E];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    if (c < ncomp) load_fwd(c, ps_[c]);
  if (P.adjoint && nop) {
    for (int o = 0; o < nop; ++o) {
      V gv[E];
      load_fwd(ncomp + o, gv);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const Kap<float> kk = kappa<float>(P, kx, ky, klayout<E>(t, j));
        for (int c = 0; c < 3; ++c)
          if (c < ncomp) ps_[c][j] = cadd(ps_[c][j], op_adjoint<float>(P.op, 3, o, c, kk, gv[j]));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const float m = multiplier<float>(P, kx, ky, klayout<E>(t, j));
    for (int c = 0; c < 3; ++c)
      if (c < ncomp) ps_[c][j] = cscale(ps_[c][j], m);
  }
  if (!P.adjoint) {
    for (int o = 0; o < nop; ++o) {
      V u[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const Kap<float> kk = kappa<float>(P, kx, ky, klayout<E>(t, j));
        V pv[3];
        for (int c = 0; c < 3; ++c) pv[c] = c < ncomp ? ps_[c][j] : czero<V>();
        u[j] = op_forward<float>(P.op, 3, o, kk, pv);
      }
      inv_store(ncomp + o, u);
    }
  }
  for (int c = 0; c < 3; ++c)
    if (c < ncomp) inv_store(c, ps_[c]);
}

// YI: 8 rows (consecutive z, fixed f and kx) of I2 along ky -> B rows along y
template <int E>
__device__ void fast_yi(const Prob<float> &P, const FastGeo &g, const FPass &ps, int tile, cx<float> *wsm) {
  typedef cx<float> V;
  constexpr int L = 32 * E;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int tz = cdiv(nuz, 8);
  const int iz = tile % tz;
  const int rest = tile / tz;
  const int kxl = rest % ps.nkx;
  const int f = rest / ps.nkx;
  const int kx = ps.kx0 + kxl;
  const int z = iz * 8 + warp;
  if (z >= nuz) return;
  const size_t slot = (size_t)ps.slot * g.nfmax * g.S * L * nuz;
  const V *src = reinterpret_cast<const V *>(P.I2) + slot + (((size_t)f * g.S + kxl) * nuz + z) * L;
  V v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = __ldcg(&src[klayout<E>(t, j)]);
  wfft_inv<float, E>(v, wsm, P.ax[1].tw);
  V *dst = reinterpret_cast<V *>(P.B) + (((size_t)f * nsx + kx) * nuz + z) * nuy;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int y = t + 32 * r;
    if (y < nuy) dst[y] = v[r];
  }
}

// persistent YZ executor over the slab work list (same queue / bounded-wait
// protocol as k_exec)
template <int E>
__global__ void __launch_bounds__(SF_FAST_THREADS)
    k_fyz(const Prob<float> *probs, FastGeo g, const FPass *passes, const int *pass_start, int npass, unsigned *done,
          ExecCtl *ctl, unsigned *sticky, unsigned long long timeout_ns, IOArgs<float> io) {
  typedef cx<float> V;
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ __align__(16) Prob<float> sP;
  __shared__ FPass sPass;
  __shared__ int s_item, s_pass, s_ok;
  load_prob<float>(sP, probs, io);
  V *wsm_all = reinterpret_cast<V *>(fsm);
  V *T = wsm_all + fast_wsm_elems<E>();
  V *wsm = wsm_all + (threadIdx.x >> 5) * E * 33;
  const int total = pass_start[npass];
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = (int)atomicAdd(&ctl->next, 1u);
      s_item = it;
      s_ok = 1;
      if (it < total) {
        int lo = 0, hi = npass - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (pass_start[mid] <= it) lo = mid;
          else hi = mid - 1;
        }
        s_pass = lo;
        sPass = passes[lo];
        for (int d = 0; d < 2 && s_ok; ++d) {
          const int dp = sPass.dep[d];
          if (dp < 0) continue;
          const unsigned need = (unsigned)sPass.depcnt[d];
          const unsigned long long t0 = global_ns();
          unsigned iters = 0;
          while (ld_acquire(&done[dp]) < need) {
            __nanosleep(64);
            if (((++iters) & 255u) == 0 && (global_ns() - t0 > timeout_ns || iters > (1u << 28))) {
              atomicCAS(&ctl->error, 0u, 6u);
              atomicExch(&ctl->err_pass, (unsigned)lo);
              atomicOr(sticky, 1u);
              s_ok = 0;
              break;
            }
          }
        }
      }
    }
    __syncthreads();
    const int it = s_item;
    if (it >= total) break;
    if (s_ok) {
      const int tile = it - pass_start[s_pass];
      switch (sPass.kind) {
        case FK_YF: fast_yf<E>(sP, g, sPass, tile, wsm, T); break;
        case FK_ZS: fast_zs<E>(sP, g, sPass, tile, wsm, T); break;
        default: fast_yi<E>(sP, g, sPass, tile, wsm); break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[s_pass], 1u);
    }
  }
}

}  // namespace sfg
