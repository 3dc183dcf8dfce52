// sf_tiles.cuh -- the passes of the solve, one tile at a time.
//
// Data flow of a 3D solve (Sec. 2.3 pencil order x -> y -> z, inverse z -> y -> x):
//   source [c][z][y][x] --XFWD--> A [c][kx][z][y]        (x transform, transposed store)
//   A  --YFWD-->  I1 [c][kx][z][ky]                        (y transform of contiguous rows)
//   I1 --ZSTAGE-> I2 [f][kx][z][ky]                        (z transform, multiply by the
//                                                           eigenvalues / Green's table,
//                                                           operator, inverse z)
//   I2 --YINV-->  B  [f][kx][z][y]                         (inverse y)
//   B  --XINV-->  result [f][z][y][x]                      (inverse x, extraction, fill)
// 2D: XFWD -> YSTAGE2 (y transform, multiply, operator, inverse y) -> XINV.
// Complex spectra (periodic / unbounded axes) store float2/double2; real
// spectra (Dirichlet / Neumann) store the real DST/DCT coefficients.
#pragma once

#include "sf_device.cuh"

namespace sfg {

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// lines per tile along the row / column passes
__host__ __device__ inline int lines_per_tile(int cpath, int W) { return cpath ? W : 2 * W; }

// ---------------------------------------------------------------------------
// generic helpers working on one shared buffer of W interleaved lines
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void zero_buf(cx<T> *a, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) a[e] = czero<cx<T>>();
}

// Place data point q of source line j at its extension position(s).
// Complex lines (periodic/unbounded) occupy a whole packed line; real lines
// are packed two per complex line (even j -> real part, odd j -> imaginary).
template <typename T> __device__ __forceinline__ void put_ext_c(cx<T> *a, const Axis<T> &ax, int Wp, int j, int q, cx<T> v) {
  a[q * Wp + j] = v;  // periodic / unbounded: position q, zero padding already in place
}
template <typename T> __device__ __forceinline__ void put_ext_r(cx<T> *a, const Axis<T> &ax, int Wp, int j, int q, T v) {
  T *af = reinterpret_cast<T *>(a);
  const int l = j >> 1, part = j & 1;
  if (ak_mixed(ax.kind)) {  // both mirrored unknowns of the doubled Dirichlet axis, each with its odd image
    int qa, qb;
    mixed_pair(ax.kind, ax.n, q, qa, qb);
    const int off = ak_mixed_regular(ax.kind) ? 1 : 0, L = ax.L;
    af[2 * ((qa + off) * Wp + l) + part] = v;
    af[2 * ((L - 1 - qa) * Wp + l) + part] = -v;
    if (qb != qa) {
      af[2 * ((qb + off) * Wp + l) + part] = v;
      af[2 * ((L - 1 - qb) * Wp + l) + part] = -v;
    }
    return;
  }
  const int m = ext_pos(ax.kind, ax.n, q);
  af[2 * (m * Wp + l) + part] = v;
  int sg;
  const int mm = ext_mirror(ax.kind, ax.n, q, sg);
  if (mm >= 0) af[2 * (mm * Wp + l) + part] = sg > 0 ? v : -v;
}
// value of data point q of line j after an inverse transform
template <typename T> __device__ __forceinline__ T get_ext_r(const cx<T> *a, const Axis<T> &ax, int Wp, int j, int q) {
  int m;
  if (ak_mixed(ax.kind)) {
    int qa, qb;
    mixed_pair(ax.kind, ax.n, q, qa, qb);
    m = qa + (ak_mixed_regular(ax.kind) ? 1 : 0);
  } else {
    m = ext_pos(ax.kind, ax.n, q);
  }
  const cx<T> v = a[m * Wp + (j >> 1)];
  return (j & 1) ? v.y : v.x;
}
// FFT index of real coefficient ci (mixed axes: the odd modes of the doubled axis)
template <typename T> __device__ __forceinline__ int coef_index(const Axis<T> &ax, int ci) {
  return ak_mixed(ax.kind) ? 2 * ci + 1 : ci + ax.k0;
}

// Real coefficient ci of real line j (packed in line j/2) from the forward FFT
// output: Hermitian split, then division by the kind's phase.
template <typename T> __device__ __forceinline__ T coef_r(const cx<T> *a, const Axis<T> &ax, int Wp, int j, int ci) {
  typedef cx<T> V;
  const int k = coef_index(ax, ci);
  const int L = ax.L;
  const int l = j >> 1;
  const V zk = a[k * Wp + l];
  const V zm = a[((L - k) % L) * Wp + l];
  V e;
  if (j & 1) {  // E_b = (Zk - conj Zm) / (2i)
    e = mk<V>((zk.y + zm.y) * (T)0.5, -(zk.x - zm.x) * (T)0.5);
  } else {  // E_a = (Zk + conj Zm) / 2
    e = mk<V>((zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5);
  }
  const V ph = ax.phase[k];
  return e.x * ph.x + e.y * ph.y;  // Re(e * conj(ph))
}

// Build the packed spectrum Z of lines (2l, 2l+1) from real coefficients:
// E_k = phase_k * c_{k-k0}, Z_k = Ea + i Eb, Z_{L-k} = conj(Ea) + i conj(Eb).
// cget(j, ci) returns the coefficient of real line j (0 if absent).
template <typename T, typename CGet>
__device__ __forceinline__ void build_spec_r(cx<T> *a, const Axis<T> &ax, int Wp, int W, CGet cget) {
  typedef cx<T> V;
  const int L = ax.L, half = L / 2;
  const bool mixed = ak_mixed(ax.kind);
  const int cnt = W * (half + 1);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int l = e % W;
    const int k = e / W;
    const int ci = mixed ? ((k & 1) ? (k >> 1) : -1) : k - ax.k0;
    V ea = czero<V>(), eb = czero<V>();
    if (ci >= 0 && ci < ax.ns) {
      const V ph = ax.phase[k];
      const T ca = cget(2 * l, ci), cb = cget(2 * l + 1, ci);
      ea = cscale(ph, ca);
      eb = cscale(ph, cb);
    }
    a[k * Wp + l] = mk<V>(ea.x - eb.y, ea.y + eb.x);
    if (k >= 1 && k <= half - 1) a[(L - k) * Wp + l] = mk<V>(ea.x + eb.y, eb.x - ea.y);
  }
}

// ---------------------------------------------------------------------------
// multiplier and operators
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T multiplier(const Prob<T> &P, int kx, int ky, int kz) {
  if (P.green) {
    int kyf = ky, kzf = kz;
    if (P.ax[1].kind == AK_U) kyf = min(ky, P.ax[1].L - ky);
    if (P.dim == 3) {
      if (P.ax[2].kind == AK_U) kzf = min(kz, P.ax[2].L - kz);
      return __ldg(&P.ghat[((size_t)kx * P.gnz + kzf) * P.gny + kyf]);
    }
    return __ldg(&P.ghat[(size_t)kx * P.gny + kyf]);
  }
  T lam = __ldg(&P.ax[0].lam[kx]) + __ldg(&P.ax[1].lam[ky]);
  if (P.dim == 3) lam += __ldg(&P.ax[2].lam[kz]);
  return lam == (T)0 ? (T)0 : P.mscale / lam;
}

// |kappa|^2 of a real-path mode (Dirichlet / Neumann axes): coefficient index ->
// FFT index -> kunit * index per axis
template <typename T> __device__ __forceinline__ T kap2_real(const Prob<T> &P, int kx, int ky, int kz) {
  const T a = P.kunit[0] * (T)coef_index(P.ax[0], kx);
  T s = a * a;
  if (P.dim >= 2) {
    const T b = P.kunit[1] * (T)coef_index(P.ax[1], ky);
    s += b * b;
  }
  if (P.dim == 3) {
    const T c = P.kunit[2] * (T)coef_index(P.ax[2], kz);
    s += c * c;
  }
  return s;
}

// wavenumbers (Nyquist zeroed) and squared wavenumbers (Nyquist kept)
template <typename T> struct Kap {
  T x, y, z, k2;
};
template <typename T> __device__ __forceinline__ Kap<T> kappa(const Prob<T> &P, int kx, int ky, int kz) {
  Kap<T> k;
  k.x = __ldg(&P.ax[0].kap[kx]);
  k.y = __ldg(&P.ax[1].kap[ky]);
  k.k2 = __ldg(&P.ax[0].kap2[kx]) + __ldg(&P.ax[1].kap2[ky]);
  if (P.dim == 3) {
    k.z = __ldg(&P.ax[2].kap[kz]);
    k.k2 += __ldg(&P.ax[2].kap2[kz]);
  } else {
    k.z = 0;
  }
  return k;
}

// operator output o from the spectra psi[c] (complex path, forward)
template <typename T> __device__ __forceinline__ cx<T> op_forward(int op, int dim, int o, const Kap<T> &k, const cx<T> *ps) {
  typedef cx<T> V;
  switch (op) {
    case OPK_GRAD: {
      const T kk = o == 0 ? k.x : (o == 1 ? k.y : k.z);
      return mul_i(cscale(ps[0], kk));
    }
    case OPK_DIV: {
      V s = cadd(cscale(ps[0], k.x), cscale(ps[1], k.y));
      if (dim == 3) s = cadd(s, cscale(ps[2], k.z));
      return mul_i(s);
    }
    case OPK_CURL: {
      if (dim == 3) {
        if (o == 0) return mul_i(csub(cscale(ps[2], k.y), cscale(ps[1], k.z)));
        if (o == 1) return mul_i(csub(cscale(ps[0], k.z), cscale(ps[2], k.x)));
        return mul_i(csub(cscale(ps[1], k.x), cscale(ps[0], k.y)));
      }
      if (o == 0) return mul_i(cscale(ps[0], k.y));
      return mul_i(cscale(ps[0], -k.x));
    }
    case OPK_NABLA: return cscale(ps[o], -k.k2);
    default: return czero<V>();
  }
}

// adjoint: contribution of the gradient g of operator output o to component c
// (the per-mode conjugate transpose of op_forward)
template <typename T> __device__ __forceinline__ cx<T> op_adjoint(int op, int dim, int o, int c, const Kap<T> &k, cx<T> g) {
  typedef cx<T> V;
  switch (op) {
    case OPK_GRAD: {  // conj(i k_o) = -i k_o, onto component 0
      const T kk = o == 0 ? k.x : (o == 1 ? k.y : k.z);
      return c == 0 ? mul_i(cscale(g, -kk)) : czero<V>();
    }
    case OPK_DIV: {  // onto component c: -i k_c g
      const T kk = c == 0 ? k.x : (c == 1 ? k.y : k.z);
      return mul_i(cscale(g, -kk));
    }
    case OPK_CURL: {
      if (dim == 3) {  // curl is self-adjoint: rows of i[k]x transposed and conjugated
        if (o == 0) return c == 1 ? mul_i(cscale(g, k.z)) : (c == 2 ? mul_i(cscale(g, -k.y)) : czero<V>());
        if (o == 1) return c == 0 ? mul_i(cscale(g, -k.z)) : (c == 2 ? mul_i(cscale(g, k.x)) : czero<V>());
        return c == 0 ? mul_i(cscale(g, k.y)) : (c == 1 ? mul_i(cscale(g, -k.x)) : czero<V>());
      }
      // 2D: u0 = i ky psi, u1 = -i kx psi
      return o == 0 ? mul_i(cscale(g, -k.y)) : mul_i(cscale(g, k.x));
    }
    case OPK_NABLA: return c == o ? cscale(g, -k.k2) : czero<V>();
    default: return czero<V>();
  }
}

// ---------------------------------------------------------------------------
// XFWD: x transform of source lines, transposed store into A[c][kx][z][y]
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_xfwd(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &X = P.ax[0], &Y = P.ax[1], &Z = P.ax[2];
  const int W = ps.W, Wp = ps.Wp, L = X.L;
  const int RL = 2 * W;  // real lines per tile
  const int nuy = P.nuy, nuz = P.nuz, nux = X.nu;
  const int ty = cdiv(nuy, RL);
  const int iy = t % ty;
  const int rest = t / ty;
  const int qz = rest % nuz;
  const int c = rest / nuz;
  const int qy0 = iy * RL;
  if (c >= P.nin) return;  // tile outside the pass (uniform over the block)
  V *a = sm, *b = sm + bufsz;
  zero_buf<T>(a, L * Wp);
  __syncthreads();
  const T *src = P.in_ptr[c];
  const int zn = P.dim == 3 ? qz + Z.u0 : 0;
  const int ndx = X.nodes, ndy = Y.nodes;
  if (src) {
    const int cnt = RL * nux;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e / nux;
      const int q = e - r * nux;
      const int qy = qy0 + r;
      if (qy >= nuy) continue;
      const int yn = qy + Y.u0, xn = q + X.u0;
      T v = src[((size_t)zn * ndy + yn) * ndx + xn];
      if (P.has_face) {  // FD2 boundary lifting (weights include 1/rhs_scale)
        if (q == 0 && P.face[0][0]) v += P.facew[0][0] * P.face[0][0][(size_t)zn * ndy + yn];
        if (q == nux - 1 && P.face[0][1]) v += P.facew[0][1] * P.face[0][1][(size_t)zn * ndy + yn];
        if (qy == 0 && P.face[1][0]) v += P.facew[1][0] * P.face[1][0][(size_t)zn * ndx + xn];
        if (qy == nuy - 1 && P.face[1][1]) v += P.facew[1][1] * P.face[1][1][(size_t)zn * ndx + xn];
        if (P.dim == 3) {
          if (qz == 0 && P.face[2][0]) v += P.facew[2][0] * P.face[2][0][(size_t)yn * ndx + xn];
          if (qz == nuz - 1 && P.face[2][1]) v += P.facew[2][1] * P.face[2][1][(size_t)yn * ndx + xn];
        }
      }
      if (P.nrw) {  // adjoint end-point weights of regular-grid Neumann face nodes
        if (nr_node(X.kind, q, nux)) v *= (T)2;
        if (nr_node(Y.kind, qy, nuy)) v *= (T)2;
        if (P.dim == 3 && nr_node(Z.kind, qz, nuz)) v *= (T)2;
      }
      put_ext_r<T>(a, X, Wp, r, q, v);
    }
  }
  __syncthreads();
  fft_lines<T, false>(a, b, X, W, Wp);
  const size_t plane = (size_t)nuz * nuy;
  if (P.cpath) {
    V *out = reinterpret_cast<V *>(P.A);
    const int nk = P.nsx;  // L/2 + 1
    const int cnt = RL * nk;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL;
      const int kx = e / RL;
      const int qy = qy0 + r;
      if (qy >= nuy) continue;
      const int l = r >> 1;
      const V zk = a[kx * Wp + l];
      const V zm = a[((L - kx) % L) * Wp + l];
      V v;
      if (r & 1) v = mk<V>((zk.y + zm.y) * (T)0.5, -(zk.x - zm.x) * (T)0.5);
      else v = mk<V>((zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5);
      out[((size_t)c * nk + kx) * plane + (size_t)qz * nuy + qy] = v;
    }
  } else {
    T *out = reinterpret_cast<T *>(P.A);
    const int nk = P.nsx;
    const int cnt = RL * nk;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL;
      const int kx = e / RL;
      const int qy = qy0 + r;
      if (qy >= nuy) continue;
      out[((size_t)c * nk + kx) * plane + (size_t)qz * nuy + qy] = coef_r<T>(a, X, Wp, r, kx);
    }
  }
}

// ---------------------------------------------------------------------------
// YFWD (3D): rows of A along y -> I1;  ZFWD-style forward-only store for set-up
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_yfwd(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &Y = P.ax[1];
  const int W = ps.W, Wp = ps.Wp, L = Y.L;
  const int RPT = lines_per_tile(P.cpath, W);
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx, nsy = P.nsy;
  const int tz = cdiv(nuz, RPT);
  const int iz = t % tz;
  const int rest = t / tz;
  const int kx = rest % nsx;
  const int c = rest / nsx;
  const int qz0 = iz * RPT;
  if (c >= P.nin) return;
  const int nl = min(RPT, nuz - qz0);
  V *a = sm, *b = sm + bufsz;
  zero_buf<T>(a, L * Wp);
  __syncthreads();
  const size_t rowbase = ((size_t)c * nsx + kx) * nuz + qz0;  // in rows
  if (P.cpath) {
    const V *in = reinterpret_cast<const V *>(P.A) + rowbase * nuy;
    const int cnt = nl * nuy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nuy, q = e - j * nuy;
      put_ext_c<T>(a, Y, Wp, j, q, __ldcg(&in[(size_t)j * nuy + q]));
    }
  } else {
    const T *in = reinterpret_cast<const T *>(P.A) + rowbase * nuy;
    const int cnt = nl * nuy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nuy, q = e - j * nuy;
      put_ext_r<T>(a, Y, Wp, j, q, __ldcg(&in[(size_t)j * nuy + q]));
    }
  }
  __syncthreads();
  fft_lines<T, false>(a, b, Y, W, Wp);
  if (P.cpath) {
    V *out = reinterpret_cast<V *>(P.I1) + rowbase * nsy;
    const int cnt = nl * nsy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nsy, k = e - j * nsy;
      __stcg(&out[(size_t)j * nsy + k], a[k * Wp + j]);
    }
  } else {
    T *out = reinterpret_cast<T *>(P.I1) + rowbase * nsy;
    const int cnt = nl * nsy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nsy, k = e - j * nsy;
      __stcg(&out[(size_t)j * nsy + k], coef_r<T>(a, Y, Wp, j, k));
    }
  }
}

// ---------------------------------------------------------------------------
// YINV (3D): inverse y transform of rows of I2 -> B
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_yinv(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &Y = P.ax[1];
  const int W = ps.W, Wp = ps.Wp, L = Y.L;
  const int RPT = lines_per_tile(P.cpath, W);
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx, nsy = P.nsy;
  const int tz = cdiv(nuz, RPT);
  const int iz = t % tz;
  const int rest = t / tz;
  const int kx = rest % nsx;
  const int f = rest / nsx;
  const int qz0 = iz * RPT;
  if (f >= P.nout) return;
  const int nl = min(RPT, nuz - qz0);
  V *a = sm, *b = sm + bufsz;
  const size_t rowbase = ((size_t)f * nsx + kx) * nuz + qz0;
  if (P.cpath) {
    const V *in = reinterpret_cast<const V *>(P.I2) + rowbase * nsy;
    const int cnt = W * L;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / L, k = e - j * L;
      a[k * Wp + j] = j < nl ? __ldcg(&in[(size_t)j * nsy + k]) : czero<V>();
    }
  } else {
    const T *in = reinterpret_cast<const T *>(P.I2) + rowbase * nsy;
    build_spec_r<T>(a, Y, Wp, W, [&](int j, int ci) -> T { return j < nl ? __ldcg(&in[(size_t)j * nsy + ci]) : (T)0; });
  }
  __syncthreads();
  fft_lines<T, true>(a, b, Y, W, Wp);
  const int cnt = nl * nuy;
  if (P.cpath) {
    V *out = reinterpret_cast<V *>(P.B) + rowbase * nuy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nuy, q = e - j * nuy;
      __stcg(&out[(size_t)j * nuy + q], a[q * Wp + j]);
    }
  } else {
    T *out = reinterpret_cast<T *>(P.B) + rowbase * nuy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int j = e / nuy, q = e - j * nuy;
      __stcg(&out[(size_t)j * nuy + q], get_ext_r<T>(a, Y, Wp, j, q));
    }
  }
}

// ---------------------------------------------------------------------------
// spectral processing shared by the 3D z-stage and the 2D y-stage
// bufs[0..ncomp) hold the forward spectra of the components; bufs[ncomp] is the
// operator buffer; *scr the FFT scratch.  kfix(l) gives (kx, ky) of line l and
// the transform axis provides the third wavenumber from the position.
// ---------------------------------------------------------------------------
template <typename T, typename KOf>
__device__ void stage_multiply_c(const Prob<T> &P, cx<T> **bufs, int nl, int W, int Wp, int L, bool zaxis, KOf kof) {
  // psi_hat = M * f_hat for every component (complex path)
  const int cnt = L * W;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int l = e % W, k = e / W;
    if (l >= nl) continue;
    int kx, ky, kz;
    kof(l, k, kx, ky, kz);
    const T m = multiplier<T>(P, kx, ky, kz);
    for (int c = 0; c < P.ncomp; ++c) bufs[c][k * Wp + l] = cscale(bufs[c][k * Wp + l], m);
  }
}

// ---------------------------------------------------------------------------
// ZSTAGE (3D) / YSTAGE2 (2D): transform, multiply, operator, inverse
// ---------------------------------------------------------------------------
// Geometry of one stage tile: nl lines of the transform axis.
//   load(c, j, q)  -> data point q of line j of input field c (complex or real)
//   store(f, j, q, v) writes data point q of line j of output field f
//   storet(t, j, n, v) writes node n of line j of y-derivative term t (2D real path)
template <typename T, bool CP, bool LINE_FAST, typename LoadC, typename LoadR, typename StoreC, typename StoreR,
          typename KOf, typename StoreT>
__device__ void run_stage(const Prob<T> &P, const Axis<T> &ax, int W, int Wp, int nl, cx<T> *sm, size_t bufsz,
                          LoadC loadc, LoadR loadr, StoreC storec, StoreR storer, KOf kof, StoreT storet) {
  typedef cx<T> V;
  const int L = ax.L;
  const int ncomp = P.ncomp;
  const bool hasop = P.op != OPK_NONE;
  V *bufs[SF_MAXF + 2];
  for (int i = 0; i < ncomp + 1; ++i) bufs[i] = sm + (size_t)i * bufsz;
  V *scr = sm + (size_t)(ncomp + 1) * bufsz;
  const int nlu = ax.nu;  // data points per line
  // ---- load + forward transform of one field into bufs[slot]
  auto fwd_field = [&](int field, int slot) {
    V *a = bufs[slot];
    zero_buf<T>(a, L * Wp);
    __syncthreads();
    const int cnt = nl * nlu;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      int j, q;
      if (LINE_FAST) { j = e % nl; q = e / nl; } else { q = e % nlu; j = e / nlu; }
      if (CP) put_ext_c<T>(a, ax, Wp, j, q, loadc(field, j, q));
      else put_ext_r<T>(a, ax, Wp, j, q, loadr(field, j, q));
    }
    __syncthreads();
    fft_lines<T, false>(bufs[slot], scr, ax, W, Wp);
  };
  // ---- inverse transform of bufs[slot] and store as output field
  auto inv_field = [&](int slot, int field) {
    fft_lines<T, true>(bufs[slot], scr, ax, W, Wp);
    const V *a = bufs[slot];
    const int cnt = nl * nlu;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      int j, q;
      if (LINE_FAST) { j = e % nl; q = e / nl; } else { q = e % nlu; j = e / nlu; }
      if (CP) storec(field, j, q, a[q * Wp + j]);
      else storer(field, j, q, get_ext_r<T>(a, ax, Wp, j, q));
    }
    __syncthreads();
  };

  if (CP) {
    const int Wl = nl;  // complex lines in the tile
    for (int c = 0; c < ncomp; ++c) fwd_field(c, c);
    if (P.adjoint && hasop) {
      for (int o = 0; o < P.nop; ++o) {
        fwd_field(ncomp + o, ncomp);
        const int cnt = L * W;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
          const int l = e % W, k = e / W;
          if (l >= Wl) continue;
          int kx, ky, kz;
          kof(l, k, kx, ky, kz);
          const Kap<T> kk = kappa<T>(P, kx, ky, kz);
          const V g = bufs[ncomp][k * Wp + l];
          for (int c = 0; c < ncomp; ++c)
            bufs[c][k * Wp + l] = cadd(bufs[c][k * Wp + l], op_adjoint<T>(P.op, P.dim, o, c, kk, g));
        }
        __syncthreads();
      }
    }
    stage_multiply_c<T>(P, bufs, Wl, W, Wp, L, true, kof);
    __syncthreads();
    if (!P.adjoint && hasop) {
      for (int o = 0; o < P.nop; ++o) {
        const int cnt = L * W;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
          const int l = e % W, k = e / W;
          V v = czero<V>();
          if (l < Wl) {
            int kx, ky, kz;
            kof(l, k, kx, ky, kz);
            const Kap<T> kk = kappa<T>(P, kx, ky, kz);
            V psv[3];
            for (int c = 0; c < ncomp && c < 3; ++c) psv[c] = bufs[c][k * Wp + l];
            v = op_forward<T>(P.op, P.dim, o, kk, psv);
          }
          bufs[ncomp][k * Wp + l] = v;
        }
        __syncthreads();
        inv_field(ncomp, ncomp + o);
      }
    }
    for (int c = 0; c < ncomp; ++c) inv_field(c, c);
  } else {
    // real path: two real lines per packed line; multiply coefficient-wise.
    // NABLA (no basis change on Dirichlet / Neumann axes) is formed here as a
    // spectral output, -|kappa|^2 psi^, in the spare buffer.  The first
    // derivatives of the other operators along the stage axis are formed here
    // too, in the spare buffer and that axis's dual basis (sine <-> cosine,
    // the same wavenumbers), and stored by node (storet); x derivatives are
    // formed from B (PK_DXINV) and 3D y derivatives by the y-inverse term
    // pass (PK_YTERM).
    const int Wl = cdiv(nl, 2);
    const bool nabla = P.op == OPK_NABLA && !P.adjoint;
    const bool nabla_adj = P.op == OPK_NABLA && P.adjoint;  // psi gradient += -|kappa|^2 (operator gradient)
    for (int c = 0; c < ncomp; ++c) {
      fwd_field(c, c);
      if (nabla_adj) fwd_field(ncomp + c, ncomp);
      V *a = bufs[c];
      V *an = bufs[ncomp];
      const int half = L / 2;
      const bool mixed = ak_mixed(ax.kind);
      const int cnt = Wl * (half + 1);
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int l = e % Wl, k = e / Wl;
        const int ci = mixed ? ((k & 1) ? (k >> 1) : -1) : k - ax.k0;
        const V zk = a[k * Wp + l];
        const V zm = a[((L - k) % L) * Wp + l];
        V ea = mk<V>((zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5);
        V eb = mk<V>((zk.y + zm.y) * (T)0.5, -(zk.x - zm.x) * (T)0.5);
        T ma = 0, mb = 0, na = 0, nb = 0;
        V ph = czero<V>();
        if (ci >= 0 && ci < ax.ns) {
          ph = ax.phase[k];
          int kx, ky, kz;
          kof(2 * l, ci, kx, ky, kz);
          ma = multiplier<T>(P, kx, ky, kz);
          if (nabla) na = -kap2_real<T>(P, kx, ky, kz);
          if (2 * l + 1 < nl) {
            kof(2 * l + 1, ci, kx, ky, kz);
            mb = multiplier<T>(P, kx, ky, kz);
            if (nabla) nb = -kap2_real<T>(P, kx, ky, kz);
          }
        }
        T ca = ea.x * ph.x + ea.y * ph.y;
        T cb = eb.x * ph.x + eb.y * ph.y;
        if (nabla_adj && ci >= 0 && ci < ax.ns) {
          const V gk = an[k * Wp + l], gm = an[((L - k) % L) * Wp + l];
          const V ga = mk<V>((gk.x + gm.x) * (T)0.5, (gk.y - gm.y) * (T)0.5);
          const V gb = mk<V>((gk.y + gm.y) * (T)0.5, -(gk.x - gm.x) * (T)0.5);
          int kx, ky, kz;
          kof(2 * l, ci, kx, ky, kz);
          ca -= kap2_real<T>(P, kx, ky, kz) * (ga.x * ph.x + ga.y * ph.y);
          if (2 * l + 1 < nl) {
            kof(2 * l + 1, ci, kx, ky, kz);
            cb -= kap2_real<T>(P, kx, ky, kz) * (gb.x * ph.x + gb.y * ph.y);
          }
        }
        ca *= ma;
        cb *= mb;
        ea = cscale(ph, ca);
        eb = cscale(ph, cb);
        a[k * Wp + l] = mk<V>(ea.x - eb.y, ea.y + eb.x);
        if (k >= 1 && k <= half - 1) a[(L - k) * Wp + l] = mk<V>(ea.x + eb.y, eb.x - ea.y);
        if (nabla) {
          const V fa = cscale(ea, na), fb = cscale(eb, nb);
          an[k * Wp + l] = mk<V>(fa.x - fb.y, fa.y + fb.x);
          if (k >= 1 && k <= half - 1) an[(L - k) * Wp + l] = mk<V>(fa.x + fb.y, fb.x - fa.y);
        }
      }
      __syncthreads();
      const int sa = P.dim - 1;  // the stage axis
      for (int st = 0; st < P.nst; ++st) {
        if (P.adjoint || P.st_comp[st] != c) continue;  // uniform over the block
        Axis<T> Dy = ax;  // the dual basis of the stage axis
        Dy.kind = P.dkind[sa];
        Dy.u0 = P.du0[sa];
        Dy.nu = P.dnu[sa];
        Dy.k0 = P.dk0[sa];
        Dy.ns = P.dns[sa];
        Dy.phase = P.dphase[sa];
        const bool dlike = ax.kind == AK_DR || ax.kind == AK_DS || ax.kind == AK_DNR || ax.kind == AK_DNS;
        const T sgn = (T)P.st_sgn[st];
        V *at = bufs[ncomp];  // the spare buffer (the FFT below may exchange it with the scratch)
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
          const int l = e % Wl, k = e / Wl;
          const int ci = mixed ? ((k & 1) ? (k >> 1) : -1) : k - ax.k0;
          const int cd = mixed ? ci : k - Dy.k0;
          V za = czero<V>(), zb = czero<V>();
          if (ci >= 0 && ci < ax.ns && cd >= 0 && cd < Dy.ns) {
            const V zk = a[k * Wp + l];
            const V zm = a[((L - k) % L) * Wp + l];
            const V ea = mk<V>((zk.x + zm.x) * (T)0.5, (zk.y - zm.y) * (T)0.5);
            const V eb = mk<V>((zk.y + zm.y) * (T)0.5, -(zk.x - zm.x) * (T)0.5);
            const V ph = ax.phase[k];
            const T kap = P.kunit[sa] * (T)k;
            const T fac = sgn * (dlike ? kap : -kap) * ((mixed && (ci & 1)) ? (T)-1 : (T)1);
            const T ca = (ea.x * ph.x + ea.y * ph.y) * fac, cb = (eb.x * ph.x + eb.y * ph.y) * fac;
            const V pd = Dy.phase[k];
            const V da = cscale(pd, ca), db = cscale(pd, cb);
            za = mk<V>(da.x - db.y, da.y + db.x);
            zb = mk<V>(da.x + db.y, db.x - da.y);
          }
          at[k * Wp + l] = za;
          if (k >= 1 && k <= half - 1) at[(L - k) * Wp + l] = zb;
        }
        __syncthreads();
        fft_lines<T, true>(bufs[ncomp], scr, Dy, W, Wp);
        const V *r = bufs[ncomp];
        const int nodes = ax.nodes;
        const int cnt2 = nl * nodes;
        for (int e = threadIdx.x; e < cnt2; e += blockDim.x) {
          int j, n;
          if (LINE_FAST) { j = e % nl; n = e / nl; } else { n = e % nodes; j = e / nodes; }
          T v = 0;
          if (n >= Dy.u0 && n < Dy.u0 + Dy.nu) v = get_ext_r<T>(r, Dy, Wp, j, n - Dy.u0);
          storet(st, j, n, v);
        }
        __syncthreads();
      }
      inv_field(c, c);
      if (nabla) inv_field(ncomp, ncomp + c);
    }
  }
}

template <typename T> __device__ void tile_zstage(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &Z = P.ax[2];
  const int W = ps.W, Wp = ps.Wp;
  const int CPT = lines_per_tile(P.cpath, W);
  const int nsx = P.nsx, nsy = P.nsy, nuz = P.nuz;
  const int ty = cdiv(nsy, CPT);
  const int iy = t % ty;
  const int kx = t / ty;
  const int ky0 = iy * CPT;
  const int nl = min(CPT, nsy - ky0);
  if (kx >= nsx) return;
  const size_t fstride = (size_t)nsx * nuz * nsy;  // elements per field
  const size_t base = (size_t)kx * nuz * nsy + ky0;
  auto kof = [&](int l, int k, int &kx_, int &ky_, int &kz_) {
    kx_ = kx;
    ky_ = ky0 + l;
    kz_ = k;
  };
  if (P.cpath) {
    const V *in = reinterpret_cast<const V *>(P.I1);
    V *out = reinterpret_cast<V *>(P.I2);
    run_stage<T, true, true>(
        P, Z, W, Wp, nl, sm, bufsz,
        [&](int f, int j, int q) -> V { return __ldcg(&in[f * fstride + base + (size_t)q * nsy + j]); },
        [&](int, int, int) -> T { return (T)0; },
        [&](int f, int j, int q, V v) { __stcg(&out[f * fstride + base + (size_t)q * nsy + j], v); },
        [&](int, int, int, T) {}, kof, [&](int, int, int, T) {});
  } else {
    const T *in = reinterpret_cast<const T *>(P.I1);
    T *out = reinterpret_cast<T *>(P.I2);
    run_stage<T, false, true>(
        P, Z, W, Wp, nl, sm, bufsz, [&](int, int, int) -> V { return czero<V>(); },
        [&](int f, int j, int q) -> T { return __ldcg(&in[f * fstride + base + (size_t)q * nsy + j]); },
        [&](int, int, int, V) {},
        [&](int f, int j, int q, T v) { __stcg(&out[f * fstride + base + (size_t)q * nsy + j], v); }, kof,
        // z-derivative terms after the psi fields, [t][kx][z node][ky]
        [&](int st, int j, int n, T v) {
          __stcg(&out[(size_t)P.ncomp * fstride + (((size_t)st * nsx + kx) * Z.nodes + n) * nsy + ky0 + j], v);
        });
  }
}

template <typename T> __device__ void tile_ystage2(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &Y = P.ax[1];
  const int W = ps.W, Wp = ps.Wp;
  const int RPT = lines_per_tile(P.cpath, W);
  const int nsx = P.nsx, nuy = P.nuy;
  const int kx0 = t * RPT;
  const int nl = min(RPT, nsx - kx0);
  const size_t fstride = (size_t)nsx * nuy;
  const size_t base = (size_t)kx0 * nuy;
  auto kof = [&](int l, int k, int &kx_, int &ky_, int &kz_) {
    kx_ = kx0 + l;
    ky_ = k;
    kz_ = 0;
  };
  if (P.cpath) {
    const V *in = reinterpret_cast<const V *>(P.A);
    V *out = reinterpret_cast<V *>(P.B);
    run_stage<T, true, false>(
        P, Y, W, Wp, nl, sm, bufsz,
        [&](int f, int j, int q) -> V { return __ldcg(&in[f * fstride + base + (size_t)j * nuy + q]); },
        [&](int, int, int) -> T { return (T)0; },
        [&](int f, int j, int q, V v) { __stcg(&out[f * fstride + base + (size_t)j * nuy + q], v); },
        [&](int, int, int, T) {}, kof, [&](int, int, int, T) {});
  } else {
    const T *in = reinterpret_cast<const T *>(P.A);
    T *out = reinterpret_cast<T *>(P.B);
    run_stage<T, false, false>(
        P, Y, W, Wp, nl, sm, bufsz, [&](int, int, int) -> V { return czero<V>(); },
        [&](int f, int j, int q) -> T { return __ldcg(&in[f * fstride + base + (size_t)j * nuy + q]); },
        [&](int, int, int, V) {},
        [&](int f, int j, int q, T v) { __stcg(&out[f * fstride + base + (size_t)j * nuy + q], v); }, kof,
        // y-derivative terms after the psi fields, [t][kx][y node]
        [&](int st, int j, int n, T v) {
          __stcg(&out[(size_t)P.ncomp * fstride + ((size_t)st * nsx + kx0 + j) * Y.nodes + n], v);
        });
  }
}

// ---------------------------------------------------------------------------
// ZFWD (set-up): forward z transform of real columns of I1, coefficients to fwd_out
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_zfwd(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &Z = P.ax[2];
  const int W = ps.W, Wp = ps.Wp, L = Z.L;
  const int CPT = 2 * W;
  const int nsx = P.nsx, nsy = P.nsy, nuz = P.nuz;
  const int ty = cdiv(nsy, CPT);
  const int iy = t % ty;
  const int kx = t / ty;
  const int ky0 = iy * CPT;
  const int nl = min(CPT, nsy - ky0);
  V *a = sm, *b = sm + bufsz;
  zero_buf<T>(a, L * Wp);
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(P.I1) + (size_t)kx * nuz * nsy + ky0;
  const int cnt = nl * nuz;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int j = e % nl, q = e / nl;
    put_ext_r<T>(a, Z, Wp, j, q, __ldcg(&in[(size_t)q * nsy + j]));
  }
  __syncthreads();
  fft_lines<T, false>(a, b, Z, W, Wp);
  T *out = P.fwd_out + (size_t)kx * Z.ns * nsy + ky0;
  const int cnt2 = nl * Z.ns;
  for (int e = threadIdx.x; e < cnt2; e += blockDim.x) {
    const int j = e % nl, k = e / nl;
    out[(size_t)k * nsy + j] = coef_r<T>(a, Z, Wp, j, k);
  }
}

// ---------------------------------------------------------------------------
// XINV: inverse x transform of 2W real lines from B (transposed read),
// extraction and store of the result; Dirichlet x-boundary nodes filled
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_xinv(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const Axis<T> &X = P.ax[0], &Y = P.ax[1], &Z = P.ax[2];
  const int W = ps.W, Wp = ps.Wp, L = X.L;
  const int RL = 2 * W;
  const int nuy = P.nuy, nuz = P.nuz, nux = X.nu, nsx = P.nsx;
  const int ty = cdiv(nuy, RL);
  const int iy = t % ty;
  const int rest = t / ty;
  const int qz = rest % nuz;
  const int f = rest / nuz;
  const int qy0 = iy * RL;
  const int nl = min(RL, nuy - qy0);
  if (f >= P.nout) return;
  V *a = sm, *stg = sm + bufsz;
  const size_t plane = (size_t)nuz * nuy;
  const size_t base = (size_t)f * nsx * plane + (size_t)qz * nuy + qy0;
  // stage the transposed block [kx][r] through shared memory
  if (P.cpath) {
    const V *in = reinterpret_cast<const V *>(P.B);
    const int cnt = nsx * RL;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL, kx = e / RL;
      stg[e] = r < nl ? __ldcg(&in[base + (size_t)kx * plane + r]) : czero<V>();
    }
    __syncthreads();
    // Z_k = A_k + i B_k (k <= L/2), Z_{L-k} = conj(A_k) + i conj(B_k); DC and Nyquist real-projected
    const int half = L / 2;
    const int cnt2 = W * (half + 1);
    for (int e = threadIdx.x; e < cnt2; e += blockDim.x) {
      const int l = e % W, k = e / W;
      V A = stg[k * RL + 2 * l], Bv = stg[k * RL + 2 * l + 1];
      if (k == 0 || k == half) {
        A.y = 0;
        Bv.y = 0;
      }
      a[k * Wp + l] = mk<V>(A.x - Bv.y, A.y + Bv.x);
      if (k >= 1 && k < half) a[(L - k) * Wp + l] = mk<V>(A.x + Bv.y, Bv.x - A.y);
    }
  } else {
    const T *in = reinterpret_cast<const T *>(P.B);
    T *stgr = reinterpret_cast<T *>(stg);
    const int cnt = nsx * RL;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL, kx = e / RL;
      stgr[e] = r < nl ? __ldcg(&in[base + (size_t)kx * plane + r]) : (T)0;
    }
    __syncthreads();
    build_spec_r<T>(a, X, Wp, W, [&](int j, int ci) -> T { return stgr[ci * RL + j]; });
  }
  __syncthreads();
  V *scr = stg;
  fft_lines<T, true>(a, scr, X, W, Wp);
  T *dst = P.out_ptr[f];
  const int zn = P.dim == 3 ? qz + Z.u0 : 0;
  const int ndx = X.nodes, ndy = Y.nodes;
  const int dmask = dnode_mask(X.kind);  // regular-grid Dirichlet face nodes of x, also written here
  const int nbd = (dmask & 1) + (dmask >> 1);
  const int nxw = nux + nbd;
  const int cnt = nl * nxw;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int r = e / nxw;
    const int p = e - r * nxw;
    const int qy = qy0 + r;
    const int yn = qy + Y.u0;
    int xn;
    T v;
    if (p >= nux) {  // boundary node x = 0 or x = n
      const int side = nbd == 2 ? p - nux : (dmask == 1 ? 0 : 1);
      xn = side == 0 ? 0 : X.n;
      v = 0;  // face data for psi; operator outputs (the series) vanish there
      if (!P.adjoint && f < P.ncomp && P.face[0][side]) v = P.face[0][side][(size_t)zn * ndy + yn];
    } else {
      xn = p + X.u0;
      v = get_ext_r<T>(a, X, Wp, r, p);
      if (P.nrw) {
        if (nr_node(X.kind, p, nux)) v *= (T)0.5;
        if (nr_node(Y.kind, qy, nuy)) v *= (T)0.5;
        if (P.dim == 3 && nr_node(Z.kind, qz, nuz)) v *= (T)0.5;
      }
    }
    dst[((size_t)zn * ndy + yn) * ndx + xn] = v;
  }
}

// ---------------------------------------------------------------------------
// FILL: regular-Dirichlet boundary planes of y and z (priority z > y > x)
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_fill(const Prob<T> &P, const Pass<T> &ps, int t) {
  const Axis<T> &X = P.ax[0], &Y = P.ax[1], &Z = P.ax[2];
  const int ndx = X.nodes, ndy = Y.nodes, ndz = P.dim == 3 ? Z.nodes : 1;
  const int ym = dnode_mask(Y.kind), zm = P.dim == 3 ? dnode_mask(Z.kind) : 0;
  const int nys = (ym & 1) + (ym >> 1), nzs = (zm & 1) + (zm >> 1);  // Dirichlet face planes per axis
  const int ny_pl = nys * ndz * ndx;
  const int nz_pl = nzs * ndy * ndx;
  const int per_field = ny_pl + nz_pl;
  const int total = per_field * P.nout;
  const int chunk = 4096;
  const int e0 = t * chunk;
  for (int e = e0 + threadIdx.x; e < min(total, e0 + chunk); e += blockDim.x) {
    const int f = e / per_field;
    int g = e - f * per_field;
    T *dst = P.out_ptr[f];
    if (g < ny_pl) {  // y planes
      const int si = g / (ndz * ndx);
      g -= si * ndz * ndx;
      const int side = nys == 2 ? si : (ym == 1 ? 0 : 1);
      const int zn = g / ndx, xn = g - zn * ndx;
      if (((zm & 1) && zn == 0) || ((zm & 2) && zn == Z.n)) continue;  // owned by the z planes
      const int yn = side == 0 ? 0 : Y.n;
      T v = 0;
      if (!P.adjoint && f < P.ncomp && P.face[1][side]) v = P.face[1][side][(size_t)zn * ndx + xn];
      dst[((size_t)zn * ndy + yn) * ndx + xn] = v;
    } else {
      g -= ny_pl;
      const int si = g / (ndy * ndx);
      g -= si * ndy * ndx;
      const int side = nzs == 2 ? si : (zm == 1 ? 0 : 1);
      const int yn = g / ndx, xn = g - yn * ndx;
      const int zn = side == 0 ? 0 : Z.n;
      T v = 0;
      if (!P.adjoint && f < P.ncomp && P.face[2][side]) v = P.face[2][side][(size_t)yn * ndx + xn];
      dst[((size_t)zn * ndy + yn) * ndx + xn] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// MULT1D: the spectral step of a 1D solve (Sec. 2.4), one thread per x mode
// over SF_MULT1D_MODES modes per tile: psi^ = m(kx) f^ with the eigenvalue or
// Green's multiplier, then the operator outputs (complex path: d/dx for GRAD
// and DIV, -kappa^2 for NABLA).  The adjoint adds the conjugate-transposed
// operator terms to the psi gradient before the (real) multiplier.
// ---------------------------------------------------------------------------
#define SF_MULT1D_MODES 256
template <typename T> __device__ void tile_mult1d(const Prob<T> &P, const Pass<T> &ps, int t) {
  typedef cx<T> V;
  const Axis<T> &X = P.ax[0];
  const int nk = P.nsx, ncomp = P.ncomp, nop = P.nop;
  for (int e = threadIdx.x; e < SF_MULT1D_MODES; e += blockDim.x) {
    const int kx = t * SF_MULT1D_MODES + e;
    if (kx >= nk) break;
    T m;
    if (P.green) {
      m = __ldg(&P.ghat[kx]);
    } else {
      const T lam = __ldg(&X.lam[kx]);
      m = lam == (T)0 ? (T)0 : P.mscale / lam;
    }
    if (P.cpath) {
      const V *A = reinterpret_cast<const V *>(P.A);
      V *B = reinterpret_cast<V *>(P.B);
      const T k = __ldg(&X.kap[kx]), k2 = __ldg(&X.kap2[kx]);
      if (!P.adjoint) {
        V psv[SF_MAXF];
        for (int c = 0; c < ncomp; ++c) {
          psv[c] = cscale(__ldcg(&A[(size_t)c * nk + kx]), m);
          __stcg(&B[(size_t)c * nk + kx], psv[c]);
        }
        for (int o = 0; o < nop; ++o) {
          const V v = P.op == OPK_NABLA ? cscale(psv[o], -k2) : mul_i(cscale(psv[0], k));
          __stcg(&B[(size_t)(ncomp + o) * nk + kx], v);
        }
      } else {
        for (int c = 0; c < ncomp; ++c) {
          V g = __ldcg(&A[(size_t)c * nk + kx]);
          for (int o = 0; o < nop; ++o) {
            const V go = __ldcg(&A[(size_t)(ncomp + o) * nk + kx]);
            if (P.op == OPK_NABLA) {
              if (o == c) g = cadd(g, cscale(go, -k2));
            } else if (c == 0) {
              g = cadd(g, mul_i(cscale(go, -k)));
            }
          }
          __stcg(&B[(size_t)c * nk + kx], cscale(g, m));
        }
      }
    } else {
      const T *A = reinterpret_cast<const T *>(P.A);
      T *B = reinterpret_cast<T *>(P.B);
      const T kap = P.kunit[0] * (T)coef_index(X, kx);
      for (int c = 0; c < ncomp; ++c) {
        T g = __ldcg(&A[(size_t)c * nk + kx]);
        if (P.op == OPK_NABLA && P.adjoint) g -= kap * kap * __ldcg(&A[(size_t)(ncomp + c) * nk + kx]);
        const T v = m * g;
        __stcg(&B[(size_t)c * nk + kx], v);
        if (P.op == OPK_NABLA && !P.adjoint) __stcg(&B[(size_t)(ncomp + c) * nk + kx], -kap * kap * v);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// DERIV: one term of an operator output on Dirichlet / Neumann axes.  Along
// axis a the solution's lines (unknown nodes) are expanded in the axis's
// basis (forward R2R), each mode is scaled by sign * kappa (order 1) or
// -kappa^2 (order 2), and the series is evaluated by the inverse R2R of the
// dual basis (order 1: sine <-> cosine; the quarter-wave pair D-N <-> N-D,
// whose doubled-axis representations differ by (-1)^m) or of the axis itself
// (order 2) at that basis's unknown nodes; every other node of the output line
// is zero, as are lines through regular Dirichlet face nodes of the other
// axes (the series vanishes there).  Only modes present in both bases are
// kept.  acc = 1 adds the term to the output instead of writing it.
// order = 3 is the transpose of the order-1 term (the adjoint): the operator
// gradient's lines are read in the dual basis, doubled on that basis's
// regular-grid Neumann face nodes, transformed, scaled by the same factor,
// inverse transformed in the axis's own basis, halved on its Neumann face
// nodes and added to the psi gradient (for these transforms F^T = V G / 2 and
// G^T = 2 F V^-1 on the shared modes, V = 2 except 1 on those face nodes).
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_deriv(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const int ax = ps.arg[0], comp = ps.arg[1], o = ps.arg[2], order = ps.arg[3], sgn = ps.arg[4], acc = ps.arg[5];
  const bool adj = order == 3;  // transpose of the first derivative: dual basis in, own basis out
  const Axis<T> &X = P.ax[ax];
  Axis<T> Dx = X;
  if (order != 2) {
    Dx.kind = P.dkind[ax];
    Dx.u0 = P.du0[ax];
    Dx.nu = P.dnu[ax];
    Dx.k0 = P.dk0[ax];
    Dx.ns = P.dns[ax];
    Dx.phase = P.dphase[ax];
  }
  const Axis<T> &Af = adj ? Dx : X;  // basis of the input lines (forward transform)
  const Axis<T> &Ai = adj ? X : Dx;  // basis of the output lines (inverse transform)
  const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;  // the other two axes, ascending
  const Axis<T> &B1 = P.ax[b1], &B2 = P.ax[b2];
  const int nd0 = P.ax[0].nodes, nd1 = P.ax[1].nodes;
  const size_t st[3] = {1, (size_t)nd0, (size_t)nd0 * nd1};
  const int nlines = B1.nodes * B2.nodes;
  const int W = ps.W, Wp = ps.Wp, RL = 2 * W, L = X.L, half = L / 2;
  const int l0 = t * RL;
  // forward: psi_comp -> operator output o; adjoint: gradient of output o -> h_comp
  const T *src = adj ? P.in_ptr[P.ncomp + o] : P.out_ptr[comp];
  T *dst = adj ? P.out_ptr[comp] : P.out_ptr[P.ncomp + o];
  auto line_base = [&](int li, bool &inside) -> size_t {
    const int u = li % B1.nodes, v = li / B1.nodes;
    inside = u >= B1.u0 && u < B1.u0 + B1.nu && v >= B2.u0 && v < B2.u0 + B2.nu;
    return (size_t)u * st[b1] + (size_t)v * st[b2];
  };
  // x derivatives walk along the contiguous lines; y and z derivatives take
  // consecutive lines (consecutive x) on consecutive threads, so that every
  // warp access covers contiguous memory
  const bool line_fast = ax != 0;
  V *a = sm, *b = sm + bufsz;
  zero_buf<T>(a, L * Wp);
  __syncthreads();
  for (int e = threadIdx.x; e < RL * Af.nu; e += blockDim.x) {
    const int r = line_fast ? e % RL : e / Af.nu;
    const int q = line_fast ? e / RL : e - r * Af.nu;
    const int li = l0 + r;
    if (li >= nlines) continue;
    bool inside;
    const size_t base = line_base(li, inside);
    if (!inside) continue;
    T v = src[base + (size_t)(q + Af.u0) * st[ax]];
    if (adj && nr_node(Af.kind, q, Af.nu)) v *= (T)2;  // transpose of the forward end-point weights
    put_ext_r<T>(a, Af, Wp, r, q, v);
  }
  __syncthreads();
  fft_lines<T, false>(a, b, Af, W, Wp);
  const bool mixed = ak_mixed(X.kind);
  const bool dlike = X.kind == AK_DR || X.kind == AK_DS || X.kind == AK_DNR || X.kind == AK_DNS;
  const T invL = (T)1 / (T)L;
  for (int e = threadIdx.x; e < W * (half + 1); e += blockDim.x) {
    const int l = e % W, k = e / W;
    const int ci = mixed ? ((k & 1) ? (k >> 1) : -1) : k - X.k0;
    const int cd = mixed ? ci : k - Dx.k0;
    V za = czero<V>(), zb = czero<V>();
    if (ci >= 0 && ci < X.ns && cd >= 0 && cd < Dx.ns) {
      const T kap = P.kunit[ax] * (T)k;
      T fac;
      if (order == 2) fac = -kap * kap * invL;
      else fac = (T)sgn * (dlike ? kap : -kap) * ((mixed && (ci & 1)) ? (T)-1 : (T)1) * invL;
      const int cf = adj ? cd : ci;
      const T ca = coef_r<T>(a, Af, Wp, 2 * l, cf) * fac, cb = coef_r<T>(a, Af, Wp, 2 * l + 1, cf) * fac;
      const V ph = Ai.phase[k];
      const V ea = cscale(ph, ca), eb = cscale(ph, cb);
      za = mk<V>(ea.x - eb.y, ea.y + eb.x);
      zb = mk<V>(ea.x + eb.y, eb.x - ea.y);
    }
    b[k * Wp + l] = za;
    if (k >= 1 && k <= half - 1) b[(L - k) * Wp + l] = zb;
  }
  __syncthreads();
  fft_lines<T, true>(b, a, Ai, W, Wp);
  for (int e = threadIdx.x; e < RL * X.nodes; e += blockDim.x) {
    const int r = line_fast ? e % RL : e / X.nodes;
    const int j = line_fast ? e / RL : e - r * X.nodes;
    const int li = l0 + r;
    if (li >= nlines) continue;
    bool inside;
    const size_t idx = line_base(li, inside) + (size_t)j * st[ax];
    T v = 0;
    if (inside && j >= Ai.u0 && j < Ai.u0 + Ai.nu) {
      v = get_ext_r<T>(b, Ai, Wp, r, j - Ai.u0);
      if (adj && nr_node(Ai.kind, j - Ai.u0, Ai.nu)) v *= (T)0.5;
    }
    if (acc) dst[idx] += v;
    else dst[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// DXINV: one derivative term of an operator output on Dirichlet / Neumann
// axes, formed where its axis is still spectral, then inverse transformed
// along x and added to (or written as) the output.
//  order 1, x derivative: from B, the x coefficients of psi_c are scaled by
//    sign * kappa, moved to the dual basis (sine <-> cosine, the same
//    wavenumbers; (-1)^m between the quarter-wave pair's doubled-axis
//    representations) and inverse transformed in that basis (the series
//    derivative of reading Z13 of Sec. 2.4.3).
//  order 4, a y or z derivative: term t of B (already inverse transformed
//    along y and z, stored by node after the psi fields of B as
//    [t][kx][z node][y node]) inverse transformed in psi's own x basis.
// Formed this way, a term's rounding scales with the term itself; a pass over
// the computed psi (PK_DERIV) weights psi's rounding by kappa.  The tile covers
// every (y, z) node line: lines through regular Dirichlet face nodes, and x
// nodes outside the basis's unknowns, are zero (the series vanishes there).
// acc = 1 adds the term.
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_dxinv(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const int src_i = ps.arg[1], o = ps.arg[2], order = ps.arg[3], sgn = ps.arg[4], acc = ps.arg[5];
  const bool yterm = order == 4;
  const Axis<T> &X = P.ax[0], &Y = P.ax[1], &Z = P.ax[2];
  Axis<T> Dx = X;  // the dual basis of x
  Dx.kind = P.dkind[0];
  Dx.u0 = P.du0[0];
  Dx.nu = P.dnu[0];
  Dx.k0 = P.dk0[0];
  Dx.ns = P.dns[0];
  Dx.phase = P.dphase[0];
  const Axis<T> &Ai = yterm ? X : Dx;  // basis of the output lines
  const int W = ps.W, Wp = ps.Wp, RL = 2 * W;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx;
  const int ndx = X.nodes;
  const int ndy = P.dim >= 2 ? Y.nodes : 1, ndz = P.dim == 3 ? Z.nodes : 1;
  const int yu0 = P.dim >= 2 ? Y.u0 : 0, zu0 = P.dim == 3 ? Z.u0 : 0;
  const int ty = cdiv(ndy, RL);
  const int iy = t % ty;
  const int zn = t / ty;
  if (zn >= ndz) return;
  const int yn0 = iy * RL;
  const int nl = min(RL, ndy - yn0);
  const int qz = zn - zu0;
  const bool zin = qz >= 0 && qz < nuz;
  V *a = sm, *stg = sm + bufsz;
  T *stgr = reinterpret_cast<T *>(stg);
  const T *in = reinterpret_cast<const T *>(P.B);
  const size_t plane = (size_t)nuz * nuy;
  // the transposed block [kx][r]: psi_c's x coefficients on the unknown y / z
  // lines, or term t's on every y node line
  const int cnt = nsx * RL;
  if (yterm) {
    const size_t base = (size_t)P.ncomp * nsx * plane + (size_t)src_i * nsx * ndz * ndy + (size_t)zn * ndy + yn0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL, kx = e / RL;
      stgr[e] = r < nl ? __ldcg(&in[base + (size_t)kx * ndz * ndy + r]) : (T)0;
    }
  } else {
    const size_t base = (size_t)src_i * nsx * plane + (size_t)(zin ? qz : 0) * nuy;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int r = e % RL, kx = e / RL;
      const int qy = yn0 + r - yu0;
      stgr[e] = (r < nl && zin && qy >= 0 && qy < nuy) ? __ldcg(&in[base + (size_t)kx * plane + qy]) : (T)0;
    }
  }
  __syncthreads();
  if (yterm) {
    build_spec_r<T>(a, X, Wp, W, [&](int j, int ci) -> T { return stgr[ci * RL + j]; });
  } else {
    const bool mixed = ak_mixed(X.kind);
    const bool dlike = X.kind == AK_DR || X.kind == AK_DS || X.kind == AK_DNR || X.kind == AK_DNS;
    build_spec_r<T>(a, Dx, Wp, W, [&](int j, int cd) -> T {
      const int k = mixed ? 2 * cd + 1 : cd + Dx.k0;  // FFT index: the same wavenumber in both bases
      const int ci = mixed ? cd : k - X.k0;
      if (ci < 0 || ci >= X.ns) return (T)0;
      const T kap = P.kunit[0] * (T)k;
      const T fac = (T)sgn * (dlike ? kap : -kap) * ((mixed && (ci & 1)) ? (T)-1 : (T)1);
      return fac * stgr[ci * RL + j];
    });
  }
  __syncthreads();
  fft_lines<T, true>(a, stg, Ai, W, Wp);
  T *dst = P.out_ptr[P.ncomp + o];
  const int cnt2 = nl * ndx;
  for (int e = threadIdx.x; e < cnt2; e += blockDim.x) {
    const int r = e / ndx;
    const int xn = e - r * ndx;
    const int yn = yn0 + r;
    const int qy = yn - yu0;
    T v = 0;
    const bool line = yterm || (zin && qy >= 0 && qy < nuy);
    if (line && xn >= Ai.u0 && xn < Ai.u0 + Ai.nu) v = get_ext_r<T>(a, Ai, Wp, r, xn - Ai.u0);
    const size_t idx = ((size_t)zn * ndy + yn) * ndx + xn;
    if (acc) dst[idx] += v;
    else dst[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// YTERM (3D, Dirichlet / Neumann axes): the y inverse of derivative term t of
// an operator output, stored by node after the psi fields of B as
// [t][kx][z node][y node] (its x inverse is a PK_DXINV pass of order 4).
//  t < nst, a z term of the z stage (in I2 after psi's fields as
//    [t][kx][z node][ky]): inverse y in psi's own y basis.
//  t >= nst, a y term: psi_c's y coefficients (I2, the unknown z rows) scaled
//    by sign * kappa and moved to the dual basis of y, inverse y in that basis
//    (reading Z13 of Sec. 2.4.3); rows through z face nodes are zero.
// y nodes outside the output basis's unknowns are zero (the series vanishes).
// ---------------------------------------------------------------------------
template <typename T> __device__ void tile_yterm(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  typedef cx<T> V;
  const int term = ps.arg[1];
  const bool yt = term >= P.nst;
  const int comp = yt ? P.yt_comp[term - P.nst] : 0;
  const T sgn = yt ? (T)P.yt_sgn[term - P.nst] : (T)0;
  const Axis<T> &Y = P.ax[1], &Z = P.ax[2];
  Axis<T> Dy = Y;  // the dual basis of y
  Dy.kind = P.dkind[1];
  Dy.u0 = P.du0[1];
  Dy.nu = P.dnu[1];
  Dy.k0 = P.dk0[1];
  Dy.ns = P.dns[1];
  Dy.phase = P.dphase[1];
  const Axis<T> &Ai = yt ? Dy : Y;  // basis of the output rows
  const int W = ps.W, Wp = ps.Wp, RPT = 2 * W;
  const int nuy = P.nuy, nuz = P.nuz, nsx = P.nsx, nsy = P.nsy;
  const int ndy = Y.nodes, ndz = Z.nodes;
  const int tz = cdiv(ndz, RPT);
  const int iz = t % tz;
  const int kx = t / tz;
  if (kx >= nsx) return;
  const int zn0 = iz * RPT;
  const int nl = min(RPT, ndz - zn0);
  V *a = sm, *b = sm + bufsz;
  const T *I2 = reinterpret_cast<const T *>(P.I2);
  // row j (z node zn0 + j) of the input coefficients, or null where it is zero
  auto row = [&](int j) -> const T * {
    if (j >= nl) return nullptr;
    const int zn = zn0 + j;
    if (!yt) return I2 + (size_t)P.ncomp * nsx * nuz * nsy + (((size_t)term * nsx + kx) * ndz + zn) * nsy;
    const int qz = zn - Z.u0;
    if (qz < 0 || qz >= nuz) return nullptr;
    return I2 + (((size_t)comp * nsx + kx) * nuz + qz) * nsy;
  };
  if (!yt) {
    build_spec_r<T>(a, Y, Wp, W, [&](int j, int ci) -> T {
      const T *r = row(j);
      return r ? __ldcg(&r[ci]) : (T)0;
    });
  } else {
    const bool mixed = ak_mixed(Y.kind);
    const bool dlike = Y.kind == AK_DR || Y.kind == AK_DS || Y.kind == AK_DNR || Y.kind == AK_DNS;
    build_spec_r<T>(a, Dy, Wp, W, [&](int j, int cd) -> T {
      const T *r = row(j);
      if (!r) return (T)0;
      const int k = mixed ? 2 * cd + 1 : cd + Dy.k0;  // FFT index: the same wavenumber in both bases
      const int ci = mixed ? cd : k - Y.k0;
      if (ci < 0 || ci >= Y.ns) return (T)0;
      const T kap = P.kunit[1] * (T)k;
      return sgn * (dlike ? kap : -kap) * ((mixed && (ci & 1)) ? (T)-1 : (T)1) * __ldcg(&r[ci]);
    });
  }
  __syncthreads();
  fft_lines<T, true>(a, b, Ai, W, Wp);
  T *out = reinterpret_cast<T *>(P.B) + (size_t)P.ncomp * nsx * nuz * nuy + ((size_t)term * nsx + kx) * ndz * ndy;
  const int cnt = nl * ndy;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int j = e / ndy, yn = e - j * ndy;
    const int zn = zn0 + j;
    const bool line = !yt || (zn - Z.u0 >= 0 && zn - Z.u0 < nuz);
    T v = 0;
    if (line && yn >= Ai.u0 && yn < Ai.u0 + Ai.nu) v = get_ext_r<T>(a, Ai, Wp, j, yn - Ai.u0);
    __stcg(&out[(size_t)zn * ndy + yn], v);
  }
}

// dispatch one tile of a pass
template <typename T> __device__ void run_tile(const Prob<T> &P, const Pass<T> &ps, int t, cx<T> *sm, size_t bufsz) {
  switch (ps.kind) {
    case PK_XFWD: tile_xfwd<T>(P, ps, t, sm, bufsz); break;
    case PK_YFWD: tile_yfwd<T>(P, ps, t, sm, bufsz); break;
    case PK_ZSTAGE: tile_zstage<T>(P, ps, t, sm, bufsz); break;
    case PK_YINV: tile_yinv<T>(P, ps, t, sm, bufsz); break;
    case PK_XINV: tile_xinv<T>(P, ps, t, sm, bufsz); break;
    case PK_YSTAGE2: tile_ystage2<T>(P, ps, t, sm, bufsz); break;
    case PK_FILL: tile_fill<T>(P, ps, t); break;
    case PK_ZFWD: tile_zfwd<T>(P, ps, t, sm, bufsz); break;
    case PK_MULT1D: tile_mult1d<T>(P, ps, t); break;
    case PK_DERIV: tile_deriv<T>(P, ps, t, sm, bufsz); break;
    case PK_DXINV: tile_dxinv<T>(P, ps, t, sm, bufsz); break;
    case PK_YTERM: tile_yterm<T>(P, ps, t, sm, bufsz); break;
    default: break;
  }
}

}  // namespace sfg
