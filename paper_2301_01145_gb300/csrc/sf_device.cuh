// sf_device.cuh -- device-side types and the shared-memory FFT engine.
//
// The solve of SailFFish (Sec. 2.4) is a chain of 1D transforms along x, y,
// z (Sec. 2.3, "successive 1D-pencils"), a point-wise spectral multiply and
// the inverse chain.  Every 1D transform here -- the periodic DFT, the
// zero-padded unbounded DFT and the DST/DCT types of Table 1 -- is carried
// out as ONE complex FFT of length L on a "virtual extension" of the data
// line that is built while the line is loaded into shared memory:
//   periodic   L = N:   the data itself
//   unbounded  L = 2N:  data followed by N zeros (Hockney-Eastwood padding)
//   DST-I/II   L = 2N:  odd extension (about a node / about a cell face)
//   DCT-I/II   L = 2N:  even extension (about a node / about a cell face)
// Two real lines are packed as the real and imaginary part of one complex
// line; the two transforms are separated afterwards with the Hermitian
// split E_a = (Z_k + conj Z_{L-k})/2, E_b = (Z_k - conj Z_{L-k})/(2i).
// For the DST/DCT types the extension's DFT equals phase_k * c_k with c_k
// the (real, FFTW-convention) transform coefficient and phase_k one of
// 1, -i, e^{i pi k/2N}, -i e^{i pi k/2N}.
//
// The FFT itself is a Stockham autosort algorithm (Van Loan, "Computational
// Frameworks for the FFT", Sec. 1.7) with radices 2, 3, 4, 8, 16 evaluated in
// registers; W lines of a tile are interleaved in shared memory as
// buf[position * Wp + line] so that consecutive threads touch consecutive
// lines (conflict-free), and two buffers are used ping-pong.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfg {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };
template <typename T> using cx = typename CT<T>::type;

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) { return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a*conj(b)
template <typename V> __device__ __forceinline__ V conjv(V a) { return mk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V czero() { return mk<V>(0, 0); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V mul_mi(V a) { return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x); }
// multiply by i
template <typename V> __device__ __forceinline__ V mul_i(V a) { return mk<V>(-a.y, a.x); }
// a + mul_mi(b) and a - mul_mi(b), written out so that the rotation stays a
// renaming of components (no rotated value is ever formed)
template <bool INV, typename V> __device__ __forceinline__ V cadd_mi(V a, V b) {
  return INV ? mk<V>(a.x - b.y, a.y + b.x) : mk<V>(a.x + b.y, a.y - b.x);
}
template <bool INV, typename V> __device__ __forceinline__ V csub_mi(V a, V b) {
  return INV ? mk<V>(a.x + b.y, a.y - b.x) : mk<V>(a.x - b.y, a.y + b.x);
}

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// Packed FP32x2 arithmetic (sm_100 and later): a complex add or subtract of
// float2 values is one instruction instead of two.  Each component is rounded
// exactly as by the scalar operation, so results are unchanged; the FFT
// butterflies are issue-bound and mostly complex adds.  These overloads are
// declared before the butterflies so that their unqualified calls bind here.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// s * a + b with one scalar s for both components
__device__ __forceinline__ float2 cfma_s(float s, float2 a, float2 b) { return __ffma2_rn(make_float2(s, s), a, b); }
#endif
template <typename V> __device__ __forceinline__ V cfma_s(decltype(V::x) s, V a, V b) {
  return mk<V>(fma(s, a.x, b.x), fma(s, a.y, b.y));
}

// ---------------------------------------------------------------------------
// radix butterflies: y_k = sum_n x_n exp(-+ 2 pi i n k / R), in place, natural order
// ---------------------------------------------------------------------------
#define SF_SQRT1_2 0.70710678118654752440084436210484903
#define SF_COS_PI8 0.92387953251128675612818318939678829
#define SF_SIN_PI8 0.38268343236508977172845998403039887
#define SF_SQRT3_2 0.86602540378443864676372317075293618

template <bool INV, typename V> __device__ __forceinline__ void dft2(V *x) {
  V t = x[0];
  x[0] = cadd(t, x[1]);
  x[1] = csub(t, x[1]);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4v(V &a0, V &a1, V &a2, V &a3) {
  const V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd_mi<INV>(t1, d);
  a3 = csub_mi<INV>(t1, d);
}

// dft4v of (a0, a1, mul_mi(a2), a3), the rotation folded into the adds
template <bool INV, typename V> __device__ __forceinline__ void dft4v_r2(V &a0, V &a1, V &a2, V &a3) {
  const V t0 = cadd_mi<INV>(a0, a2), t1 = csub_mi<INV>(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd_mi<INV>(t1, d);
  a3 = csub_mi<INV>(t1, d);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V *x) { dft4v<INV>(x[0], x[1], x[2], x[3]); }

template <bool INV, typename V> __device__ __forceinline__ void dft3(V *x) {
  typedef decltype(V::x) T;
  V t = cadd(x[1], x[2]);
  V d = csub(x[1], x[2]);
  // y1,2 = x0 - t/2 +- (-+ i sqrt3/2) (x1 - x2)
  const V u = cscale(d, (T)SF_SQRT3_2);
  const V m = cfma_s<V>((T)-0.5, t, x[0]);
  x[0] = cadd(x[0], t);
  x[1] = cadd_mi<INV>(m, u);
  x[2] = csub_mi<INV>(m, u);
}

template <bool INV, typename V> __device__ __forceinline__ V w8(V a, int j) {  // a * exp(-+ 2 pi i j / 8), j = 0..3
  typedef decltype(V::x) T;
  const T s = (T)SF_SQRT1_2;
  switch (j) {
    case 1: return INV ? mk<V>(s * (a.x - a.y), s * (a.x + a.y)) : mk<V>(s * (a.x + a.y), s * (a.y - a.x));
    case 2: return mul_mi<INV>(a);
    case 3: return INV ? mk<V>(-s * (a.x + a.y), s * (a.x - a.y)) : mk<V>(s * (a.y - a.x), -s * (a.x + a.y));
    default: return a;
  }
}

template <bool INV, typename V> __device__ __forceinline__ void dft8(V *x) {
  // decimation in time: E = DFT4(even), O = DFT4(odd), y_k = E_k + w^k O_k
  V e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  V o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4v<INV>(e0, e1, e2, e3);
  dft4v<INV>(o0, o1, o2, o3);
  o1 = w8<INV>(o1, 1);
  o3 = w8<INV>(o3, 3);
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = cadd_mi<INV>(e2, o2); x[6] = csub_mi<INV>(e2, o2);  // w8^2 = -+i
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

template <bool INV, typename V> __device__ __forceinline__ V w16(V a, int j) {  // a * exp(-+ 2 pi i j/16), j = 0..9
  typedef decltype(V::x) T;
  // c_j = cos(2 pi j / 16), s_j = sin(2 pi j / 16)
  T c, s;
  switch (j) {
    case 0: return a;
    case 1: c = (T)SF_COS_PI8; s = (T)SF_SIN_PI8; break;
    case 2: c = (T)SF_SQRT1_2; s = (T)SF_SQRT1_2; break;
    case 3: c = (T)SF_SIN_PI8; s = (T)SF_COS_PI8; break;
    case 4: return mul_mi<INV>(a);
    case 6: c = -(T)SF_SQRT1_2; s = (T)SF_SQRT1_2; break;
    case 9: c = -(T)SF_COS_PI8; s = -(T)SF_SIN_PI8; break;
    default: c = 1; s = 0; break;
  }
  // forward: a * (c - i s); inverse: a * (c + i s)
  if (INV) return mk<V>(a.x * c - a.y * s, a.x * s + a.y * c);
  return mk<V>(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <bool INV, typename V> __device__ __forceinline__ void dft16(V *x) {
  // 16 = 4 x 4: F_s = DFT4(x_s, x_{s+4}, x_{s+8}, x_{s+12}); y_{k1+4k2} = DFT4_s(w16^{s k1} F_s[k1])
  V f[16];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    V a0 = x[s], a1 = x[s + 4], a2 = x[s + 8], a3 = x[s + 12];
    dft4v<INV>(a0, a1, a2, a3);
    f[s * 4 + 0] = a0; f[s * 4 + 1] = a1; f[s * 4 + 2] = a2; f[s * 4 + 3] = a3;
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    V t0 = f[0 * 4 + k1];
    V t1 = w16<INV>(f[1 * 4 + k1], 1 * k1);
    V t3 = w16<INV>(f[3 * 4 + k1], 3 * k1);
    if (k1 == 2) {
      dft4v_r2<INV>(t0, t1, f[2 * 4 + k1], t3);  // w16^4 = -+i
      x[k1] = t0; x[k1 + 4] = t1; x[k1 + 8] = f[2 * 4 + k1]; x[k1 + 12] = t3;
    } else {
      V t2 = w16<INV>(f[2 * 4 + k1], 2 * k1);
      dft4v<INV>(t0, t1, t2, t3);
      x[k1] = t0; x[k1 + 4] = t1; x[k1 + 8] = t2; x[k1 + 12] = t3;
    }
  }
}

template <int R, bool INV, typename V> __device__ __forceinline__ void dftR(V *x) {
  if (R == 2) dft2<INV>(x);
  else if (R == 3) dft3<INV>(x);
  else if (R == 4) dft4<INV>(x);
  else if (R == 8) dft8<INV>(x);
  else if (R == 16) dft16<INV>(x);
}

// ---------------------------------------------------------------------------
// problem description (device copy)
// ---------------------------------------------------------------------------
enum AxisKind : int {
  AK_P = 0, AK_U = 1, AK_DR = 2, AK_NR = 3, AK_DS = 4, AK_NS = 5,
  // one Dirichlet and one Neumann face (lower, upper), regular / staggered grid
  AK_DNR = 6, AK_DNS = 7, AK_NDR = 8, AK_NDS = 9
};

// An axis with a Dirichlet and a Neumann face is solved as the Dirichlet axis
// of twice the length whose data are mirrored about the Neumann face (the
// discrete problem with homogeneous Neumann data at the face is exactly the
// symmetric half of it).  Its FFT has length L = 4n; only the odd modes of the
// doubled axis (the quarter-wave modes k + 1/2) carry coefficients.
__host__ __device__ inline bool ak_mixed(int kind) { return kind >= AK_DNR; }
__host__ __device__ inline bool ak_mixed_regular(int kind) { return kind == AK_DNR || kind == AK_NDR; }
// unknown indices (qa, qb) of the doubled Dirichlet axis that hold data index q
// (qa is the one inside the original half; qb its mirror image, = qa on the Neumann node)
__host__ __device__ inline void mixed_pair(int kind, int n, int q, int &qa, int &qb) {
  switch (kind) {
    case AK_DNR: qa = q; qb = 2 * n - 2 - q; break;
    case AK_DNS: qa = q; qb = 2 * n - 1 - q; break;
    case AK_NDR: qa = n - 1 + q; qb = n - 1 - q; break;
    default: qa = n + q; qb = n - 1 - q; break;  // AK_NDS
  }
}
// regular-grid Dirichlet face nodes of an axis: bit 0 lower face, bit 1 upper face
__host__ __device__ inline int dnode_mask(int kind) {
  return kind == AK_DR ? 3 : (kind == AK_DNR ? 1 : (kind == AK_NDR ? 2 : 0));
}
// data index q is a regular-grid Neumann face node (weight 1/2 in the discrete
// orthogonality of its transform; used by the adjoint's end-point weights)
__host__ __device__ inline bool nr_node(int kind, int q, int nu) {
  return (kind == AK_NR && (q == 0 || q == nu - 1)) || (kind == AK_DNR && q == nu - 1) || (kind == AK_NDR && q == 0);
}
enum OpKind : int { OPK_NONE = 0, OPK_GRAD = 1, OPK_DIV = 2, OPK_CURL = 3, OPK_NABLA = 4 };
enum PassKind : int {
  PK_XFWD = 0,     // x transform of the source lines, transposed store to A
  PK_YFWD = 1,     // y transform of rows of A -> I1 (3D)
  PK_ZSTAGE = 2,   // z transform, multiply, operator, inverse z (3D): I1 -> I2
  PK_YINV = 3,     // inverse y transform of rows of I2 -> B (3D)
  PK_XINV = 4,     // inverse x transform, extraction and store of the result
  PK_YSTAGE2 = 5,  // 2D: y transform, multiply, operator, inverse y: A -> B
  PK_FILL = 6,     // Dirichlet boundary-plane fill of psi (regular grids)
  PK_ZFWD = 7,     // forward-only z transform (Green's table set-up): I1 -> fwd_out
  PK_MULT1D = 8,   // 1D: multiply and operator in x-spectral space: A -> B
  PK_DERIV = 9,    // Dirichlet / Neumann axes: one derivative term of an operator output
};

template <typename T> struct Axis {
  int kind;   // AxisKind
  int n;      // cells N_c
  int nodes;  // extent of the user array along this axis
  int u0;     // first unknown node
  int nu;     // number of unknowns (data points transformed)
  int L;      // FFT length
  int ns;     // number of spectral coefficients kept along this axis
  int k0;     // FFT index of coefficient 0 (real kinds: 1 for Dirichlet, 0 otherwise)
  int nst;    // number of radix stages
  int radix[5];
  const cx<T> *tw;     // exp(-2 pi i j / L), j < L
  const cx<T> *twf;    // warp-FFT twiddles, lane-contiguous (L = 256, 512; see sf_fast.cuh), else null
  const cx<T> *phase;  // real kinds: phase_k, k in [0, n]
  const T *lam;        // eigenvalue per coefficient index (bounded)
  const T *kap;        // derivative wavenumber per coefficient index, Nyquist zeroed
  const T *kap2;       // squared wavenumber per coefficient index, Nyquist kept
};

#define SF_MAXF 6

template <typename T> struct Prob {
  int dim, ncomp, nop;
  int nin, nout;  // fields entering the x transform / leaving the stage
  int cpath;      // 1: periodic/unbounded (complex spectra); 0: Dirichlet/Neumann (real)
  int op;         // OpKind
  int opc[3][3];  // operator coefficient of component c in output o: 0, +-1 (+-i kappa_axis), 2 (-|kappa|^2)
  int opa[3][3];  // axis of the derivative coefficient
  int green;      // 1: multiply by the Green's table
  int adjoint;    // 1: transposed solve
  int nrw;        // adjoint: apply regular-Neumann end-point weights
  Axis<T> ax[3];
  T rhs_scale;
  T mscale;  // eigenvalue path: rhs_scale / prod(L)
  const T *in_ptr[SF_MAXF];
  T *out_ptr[SF_MAXF];
  const T *face[3][2];
  T facew[3][2];
  int has_face;
  void *A, *I1, *I2, *B;
  const T *ghat;    // unbounded: [kx][kz][ky] octant (3D) / [kx][ky] (2D), pre-scaled
  const T *ghat_t;  // the same table as [kx][ky][kz] (register fast path)
  T *fwd_out;     // set-up: forward-only output
  // derived extents
  int nsx, nuy, nuz, nsy, nsz;
  int gny, gnz;  // Green's table extents along y, z
  int fill_count;
  // operators on Dirichlet / Neumann axes: the dual basis of each axis (sine <->
  // cosine, same length and modes) and the wavenumber of FFT index 1
  int dkind[3], du0[3], dnu[3], dk0[3], dns[3];
  const cx<T> *dphase[3];
  T kunit[3];
};

template <typename T> struct Pass {
  int kind;
  int prob;
  int ntiles;
  int W;      // packed lines per tile
  int Wp;     // padded line stride in shared memory
  int nbuf;   // shared buffers used
  int bufsz;  // complex elements per shared buffer
  int dep[2];
  int depcnt[2];
  int arg[6];  // PK_DERIV: axis, psi component, output, order (1, 2), sign, accumulate
};

// executor control block (device)
struct ExecCtl {
  unsigned int next;      // work-queue head
  unsigned int error;     // SF_ERR_* code of the first failure (0 = ok)
  unsigned int err_pass;  // pass that timed out
  unsigned int pad;
  // tracing: per pass kind (index = kind, up to 8 kinds), summed over CTAs, nanoseconds
  unsigned long long busy_ns[8];  // time between the start and the end of a tile
  unsigned long long wait_ns[8];  // time spent waiting for dependencies before a tile
  unsigned long long tiles[8];
};

// ---------------------------------------------------------------------------
// Stockham radix stage: in (L x W lines, stride Wp) -> out
// ---------------------------------------------------------------------------
template <typename T, int R, bool INV>
__device__ __forceinline__ void stockham_stage(const cx<T> *__restrict__ in, cx<T> *__restrict__ out, int L, int W, int Wp,
                                               int Ns, const cx<T> *__restrict__ tw) {
  typedef cx<T> V;
  const int nb = L / R;
  const int total = nb * W;
  const int tws = L / (Ns * R);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = b % W;
    const int j = b / W;
    const int k = j % Ns;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[(j + r * nb) * Wp + line];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = __ldg(&tw[r * k * tws]);
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    dftR<R, INV>(v);
    const int o = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[(o + r * Ns) * Wp + line] = v[r];
  }
}

// Runs the full FFT of W interleaved lines of length ax.L held in *a (scratch
// *b).  The caller has synchronised before; the result is synchronised on
// return and *a / *b are swapped so that *a holds it.
template <typename T, bool INV>
__device__ void fft_lines(cx<T> *&a, cx<T> *&b, const Axis<T> &ax, int W, int Wp) {
  int Ns = 1;
  const int L = ax.L;
  for (int s = 0; s < ax.nst; ++s) {
    const int R = ax.radix[s];
    switch (R) {
      case 16: stockham_stage<T, 16, INV>(a, b, L, W, Wp, Ns, ax.tw); break;
      case 8: stockham_stage<T, 8, INV>(a, b, L, W, Wp, Ns, ax.tw); break;
      case 4: stockham_stage<T, 4, INV>(a, b, L, W, Wp, Ns, ax.tw); break;
      case 3: stockham_stage<T, 3, INV>(a, b, L, W, Wp, Ns, ax.tw); break;
      default: stockham_stage<T, 2, INV>(a, b, L, W, Wp, Ns, ax.tw); break;
    }
    __syncthreads();
    cx<T> *t = a;
    a = b;
    b = t;
    Ns *= R;
  }
}

// ---------------------------------------------------------------------------
// extension maps (data index q <-> FFT position m) for the six axis kinds
// ---------------------------------------------------------------------------
// primary FFT position of data index q and, if any, its mirrored position
// (sign -1 for the odd extensions)
__device__ __forceinline__ int ext_pos(int kind, int n, int q) {
  return kind == AK_DR ? q + 1 : q;
}
__device__ __forceinline__ int ext_mirror(int kind, int n, int q, int &sign) {
  switch (kind) {
    case AK_DR: sign = -1; return 2 * n - 1 - q;  // position 2n - (q+1)
    case AK_NR: sign = 1; return (q >= 1 && q <= n - 1) ? 2 * n - q : -1;
    case AK_DS: sign = -1; return 2 * n - 1 - q;
    case AK_NS: sign = 1; return 2 * n - 1 - q;
    default: sign = 1; return -1;
  }
}

}  // namespace sfg
