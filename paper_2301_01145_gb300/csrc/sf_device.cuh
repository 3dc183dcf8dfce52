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

// asynchronous global -> shared copies (4 bytes each), completed by cp_async_wait_all
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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
  PK_DXINV = 10,   // Dirichlet / Neumann axes: a derivative term's inverse x into the output
  PK_YTERM = 11,   // Dirichlet / Neumann axes (3D): a derivative term's inverse y into B
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
#define SF_MAXYT 4  // derivative terms of one kind along one axis (at most one per component and output)

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
  // first-derivative terms of the operator outputs along the stage axis (y in
  // 2D, z in 3D), formed in the spectral stage in that axis's dual basis and
  // stored by node after the psi fields of the stage's output (B in 2D as
  // [t][kx][y node], I2 in 3D as [t][kx][z node][ky])
  int nst;
  int st_comp[SF_MAXYT], st_sgn[SF_MAXYT];
  // 3D: y-derivative terms, formed by the y-inverse term pass from psi's y
  // coefficients in I2; B holds every 3D term after the psi fields as
  // [t][kx][z node][y node], the stage terms first
  int n3yt;
  int yt_comp[SF_MAXYT], yt_sgn[SF_MAXYT];
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
  int arg[6];  // PK_DERIV / PK_DXINV: axis, psi component, output, order (1, 2, 3), sign, accumulate
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
// ---------------------------------------------------------------------------
// warp FFT of one line of L = 32 E points held by one warp (E = 8, 16):
// E-point DFT in registers, twiddle, one transpose through the warp's padded
// shared buffer, E-point DFT, then a radix-2 network over the G = 32 / E lanes
// of a group.  Used by the register fast path and, for FP32 lines of 256 or
// 512 points, by the general engine's fft_lines.
// ---------------------------------------------------------------------------
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

// W_32^m = exp(-2 pi i m / 32) for a compile-time m (folded to immediates
// after unrolling): cos(2 pi r / 32), r = 0..8, and quadrant symmetry
__host__ __device__ constexpr float cos32(int r) {
  return r == 0 ? 1.0f
       : r == 1 ? 0.980785280403230449126f
       : r == 2 ? 0.923879532511286756128f
       : r == 3 ? 0.831469612302545237078f
       : r == 4 ? 0.707106781186547524401f
       : r == 5 ? 0.555570233019602224742f
       : r == 6 ? 0.382683432365089771728f
       : r == 7 ? 0.195090322016128267848f
                : 0.0f;
}
template <typename V> __device__ __forceinline__ V w32c(int m) {
  m &= 31;
  float c, sn;  // cos and sin of 2 pi m / 32
  if (m <= 8) { c = cos32(m); sn = cos32(8 - m); }
  else if (m <= 16) { c = -cos32(16 - m); sn = cos32(m - 8); }
  else if (m <= 24) { c = -cos32(m - 16); sn = -cos32(24 - m); }
  else { c = cos32(32 - m); sn = -cos32(m - 24); }
  return mk<V>(c, -sn);
}
// twiddle W_L^{q j E} = W_32^{q j} of the E-point stage (L = 32 E, lane group index q < G)
template <int G, typename V> __device__ __forceinline__ V w_stage2(int q, int j) {
  if (G == 1) return w32c<V>(0);
  if (G == 2) return q ? w32c<V>(j) : w32c<V>(0);
  return q == 0 ? w32c<V>(0) : (q == 1 ? w32c<V>(j) : (q == 2 ? w32c<V>(2 * j) : w32c<V>(3 * j)));
}

// derivative wavenumber of FFT index k on a periodic or doubled axis of
// length L: ks * kappa_1 with ks = k (k < L/2), k - L (k > L/2), 0 (Nyquist),
// where kappa_1 = kap[1] of the axis; equals the kap table to one rounding
template <int L> __device__ __forceinline__ float kap_of(int k, float kap1) {
  const int ks = k < L / 2 ? k : (k > L / 2 ? k - L : 0);
  return (float)ks * kap1;
}

// k index held in register j by this lane after a forward warp FFT
template <int E> __device__ __forceinline__ int klayout(int lane, int j) {
  constexpr int G = 32 / E;
  const int k1 = lane / G, q = lane % G;
  return k1 + E * (j + E * bitrev_lanes(q, G));
}

// row stride of the warp transpose buffer: 32 + G makes (k1 * stride + q) mod 16
// a permutation over a half warp (8-byte elements), i.e. no bank conflicts
template <int E> __host__ __device__ constexpr int wrow() { return 32 + 32 / E; }
// Row of spectral index k in a 16-line transpose tile: stride 17, and the G
// lane groups of the k layout (k / E^2) shifted by E/2 slots so that a half
// warp writing one register of every lane hits 16 distinct bank pairs.
template <int E> __device__ __forceinline__ int trow(int k) { return k * 17 + (k / (E * E)) * (E / 2); }
template <int E> __host__ __device__ constexpr int trows_elems() { return 32 * E * 17 + 16; }

// ---- pruned E-point DFTs ----------------------------------------------------
// dft4 of (a0, a1, 0, 0)
template <bool INV, typename V> __device__ __forceinline__ void dft4_2in(V a0, V a1, V &y0, V &y1, V &y2, V &y3) {
  y0 = cadd(a0, a1);
  y1 = cadd_mi<INV>(a0, a1);
  y2 = csub(a0, a1);
  y3 = csub_mi<INV>(a0, a1);
}

// inputs x[E/2 .. E) are zero
template <int E, bool INV, typename V> __device__ __forceinline__ void dft_halfin(V *x) {
  if (E == 16) {
    V f[16];
#pragma unroll
    for (int s = 0; s < 4; ++s) dft4_2in<INV>(x[s], x[s + 4], f[s * 4 + 0], f[s * 4 + 1], f[s * 4 + 2], f[s * 4 + 3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      V t0 = f[k1];
      V t1 = w16<INV>(f[4 + k1], k1);
      V t3 = w16<INV>(f[12 + k1], 3 * k1);
      if (k1 == 2) {
        V t2 = f[8 + k1];
        dft4v_r2<INV>(t0, t1, t2, t3);  // w16^4 = -+i
        x[k1] = t0; x[k1 + 4] = t1; x[k1 + 8] = t2; x[k1 + 12] = t3;
      } else {
        V t2 = w16<INV>(f[8 + k1], 2 * k1);
        dft4v<INV>(t0, t1, t2, t3);
        x[k1] = t0; x[k1 + 4] = t1; x[k1 + 8] = t2; x[k1 + 12] = t3;
      }
    }
  } else {  // E == 8
    V e0, e1, e2, e3, o0, o1, o2, o3;
    dft4_2in<INV>(x[0], x[2], e0, e1, e2, e3);
    dft4_2in<INV>(x[1], x[3], o0, o1, o2, o3);
    o1 = w8<INV>(o1, 1);
    o3 = w8<INV>(o3, 3);
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
    x[2] = cadd_mi<INV>(e2, o2); x[6] = csub_mi<INV>(e2, o2);  // w8^2 = -+i
    x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
  }
}

// only outputs y[0 .. E/2) are needed
template <int E, bool INV, typename V> __device__ __forceinline__ void dft_halfout(V *x) {
  if (E == 16) {
    V f[16];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      V a0 = x[s], a1 = x[s + 4], a2 = x[s + 8], a3 = x[s + 12];
      dft4v<INV>(a0, a1, a2, a3);
      f[s * 4 + 0] = a0; f[s * 4 + 1] = a1; f[s * 4 + 2] = a2; f[s * 4 + 3] = a3;
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      const V t0 = f[k1];
      const V t1 = w16<INV>(f[4 + k1], k1);
      const V t3 = w16<INV>(f[12 + k1], 3 * k1);
      if (k1 == 2) {  // w16^4 = -+i
        const V t2 = f[8 + k1];
        x[k1] = cadd(cadd_mi<INV>(t0, t2), cadd(t1, t3));
        x[k1 + 4] = cadd_mi<INV>(csub_mi<INV>(t0, t2), csub(t1, t3));
      } else {
        const V t2 = w16<INV>(f[8 + k1], 2 * k1);
        x[k1] = cadd(cadd(t0, t2), cadd(t1, t3));
        x[k1 + 4] = cadd_mi<INV>(csub(t0, t2), csub(t1, t3));
      }
    }
  } else {
    V e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    V o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4v<INV>(e0, e1, e2, e3);
    dft4v<INV>(o0, o1, o2, o3);
    x[0] = cadd(e0, o0);
    x[1] = cadd(e1, w8<INV>(o1, 1));
    x[2] = cadd_mi<INV>(e2, o2);  // w8^2 = -+i
    x[3] = cadd(e3, w8<INV>(o3, 3));
  }
}

// ---- warp FFTs -------------------------------------------------------------
// M independent lines per warp, interleaved step by step so that their
// dependency chains overlap (wsm: M consecutive buffers of E*33 elements).
// Twiddles come from the lane-contiguous table twf of the axis:
//   twf[k1 * 32 + t]          = W_L^{t k1}       (step 1, one 256-byte row per k1)
//   twf[L + j * G + q]        = W_L^{q j E}      (step 3, E-point stage; with G = 2 the kernels
//                                                 use the equal constants W_32^{q j} of w_stage2)
//   twf[L + 32 + mm - 1 + r]  = W_{2 mm}^r       (step 3, lane stage mm)
template <typename T, int E, bool HALFIN, int M>
__device__ __forceinline__ void wfft_fwd_m(cx<T> (&v)[M][E], cx<T> *wsm, const cx<T> *__restrict__ tw) {
  typedef cx<T> V;
  constexpr int L = 32 * E, G = 32 / E, P = wrow<E>();
  const int t = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    if (HALFIN) dft_halfin<E, false>(v[m]);
    else dftR<E, false>(v[m]);
  }
  {
    // W_L^{t k1}: rows k1 < 4 and k1 = 0 mod 4 are loaded, the others are one
    // product W_L^{t (k1 & ~3)} W_L^{t (k1 & 3)} (one rounding more)
    const V w1 = __ldg(&tw[1 * 32 + t]), w2 = __ldg(&tw[2 * 32 + t]), w3 = __ldg(&tw[3 * 32 + t]);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
      V w;
      if ((k1 & 3) == 0 || k1 < 4) w = __ldg(&tw[k1 * 32 + t]);
      else {
        const V a = __ldg(&tw[(k1 & ~3) * 32 + t]);
        const int b = k1 & 3;
        w = cmul(a, b == 1 ? w1 : (b == 2 ? w2 : w3));
      }
#pragma unroll
      for (int m = 0; m < M; ++m) v[m][k1] = cmul(v[m][k1], w);
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) wsm[m * E * P + k1 * P + t] = v[m][k1];
  __syncwarp();
  const int k1 = t / G, q = t % G;
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int s = 0; s < E; ++s) v[m][s] = wsm[m * E * P + k1 * P + G * s + q];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < M; ++m) dftR<E, false>(v[m]);
#pragma unroll
  for (int j = 1; j < E; ++j) {
    // two lanes per group: constants and one select; more lanes: one table load
    const V w = G == 2 ? w_stage2<G, V>(q, j) : __ldg(&tw[L + j * G + q]);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m][j] = cmul(v[m][j], w);
  }
#pragma unroll
  for (int mm = G / 2; mm >= 1; mm >>= 1) {
    const float sg = (q & mm) ? -1.f : 1.f;  // hi lane: partner - mine, lo lane: mine + partner
    const V w = __ldg(&tw[L + 32 + mm - 1 + (q & (mm - 1))]);
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const V p = shfl_xor_c(v[m][j], mm);
        V r = cfma_s<V>(sg, v[m][j], p);
        if (mm > 1 && (q & mm)) r = cmul(r, w);
        v[m][j] = r;
      }
  }
}

template <typename T, int E, bool HALFOUT, int M>
__device__ __forceinline__ void wfft_inv_m(cx<T> (&v)[M][E], cx<T> *wsm, const cx<T> *__restrict__ tw) {
  typedef cx<T> V;
  constexpr int L = 32 * E, G = 32 / E, P = wrow<E>();
  const int t = threadIdx.x & 31;
  const int k1 = t / G, q = t % G;
#pragma unroll
  for (int mm = 1; mm < G; mm <<= 1) {
    const bool hi = (q & mm) != 0;
    const float sg = hi ? -1.f : 1.f;
    const V w = __ldg(&tw[L + 32 + mm - 1 + (q & (mm - 1))]);
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        // pair (a = lo value, b = hi value): lo <- a + conj(w) b, hi <- a - conj(w) b.
        // The hi lane twiddles its own value before the exchange.
        V mine = v[m][j];
        if (mm > 1 && hi) mine = cmulc(mine, w);
        const V p = shfl_xor_c(mine, mm);
        v[m][j] = cfma_s<V>(sg, mine, p);  // hi: p - mine, lo: p + mine
      }
  }
#pragma unroll
  for (int j = 1; j < E; ++j) {
    const V w = G == 2 ? w_stage2<G, V>(q, j) : __ldg(&tw[L + j * G + q]);
#pragma unroll
    for (int m = 0; m < M; ++m) v[m][j] = cmulc(v[m][j], w);
  }
#pragma unroll
  for (int m = 0; m < M; ++m) dftR<E, true>(v[m]);
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int s = 0; s < E; ++s) wsm[m * E * P + k1 * P + G * s + q] = v[m][s];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int kk = 0; kk < E; ++kk) v[m][kk] = wsm[m * E * P + kk * P + t];
  __syncwarp();
  {
    // conjugate of W_L^{t kk}, built as in the forward transform
    const V w1 = __ldg(&tw[1 * 32 + t]), w2 = __ldg(&tw[2 * 32 + t]), w3 = __ldg(&tw[3 * 32 + t]);
#pragma unroll
    for (int kk = 1; kk < E; ++kk) {
      V w;
      if ((kk & 3) == 0 || kk < 4) w = __ldg(&tw[kk * 32 + t]);
      else {
        const V a = __ldg(&tw[(kk & ~3) * 32 + t]);
        const int b = kk & 3;
        w = cmul(a, b == 1 ? w1 : (b == 2 ? w2 : w3));
      }
#pragma unroll
      for (int m = 0; m < M; ++m) v[m][kk] = cmulc(v[m][kk], w);
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    if (HALFOUT) dft_halfout<E, true>(v[m]);
    else dftR<E, true>(v[m]);
  }
}

// fft_lines for FP32 lines of L = 256 / 512 points with at least 8 lines per
// tile: one warp per line through the warp FFT instead of the shared-memory
// Stockham stages (no CTA barrier between radix stages).  Natural order in
// and out, like the Stockham path; the warp buffers live in the scratch *b
// (L * Wp >= 8 E wrow elements when W >= 8).  The result stays in *a.
template <int E, bool INV>
__device__ void fft_lines_warp(cx<float> *a, cx<float> *b, const Axis<float> &ax, int W, int Wp) {
  typedef cx<float> V;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  V *wsm = b + warp * E * wrow<E>();
  for (int l = warp; l < W; l += nwarps) {
    V v[1][E];
    if (!INV) {
#pragma unroll
      for (int r = 0; r < E; ++r) v[0][r] = a[(t + 32 * r) * Wp + l];
      wfft_fwd_m<float, E, false, 1>(v, wsm, ax.twf);
#pragma unroll
      for (int j = 0; j < E; ++j) a[klayout<E>(t, j) * Wp + l] = v[0][j];
    } else {
#pragma unroll
      for (int j = 0; j < E; ++j) v[0][j] = a[klayout<E>(t, j) * Wp + l];
      wfft_inv_m<float, E, false, 1>(v, wsm, ax.twf);
#pragma unroll
      for (int r = 0; r < E; ++r) a[(t + 32 * r) * Wp + l] = v[0][r];
    }
    __syncwarp();  // the warp buffer is reused by the next line
  }
  __syncthreads();
}

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
  if constexpr (sizeof(T) == 4) {
    if (ax.twf != nullptr && W >= 8 && blockDim.x == 256) {
      if (ax.L == 512) return fft_lines_warp<16, INV>(a, b, ax, W, Wp);
      if (ax.L == 256) return fft_lines_warp<8, INV>(a, b, ax, W, Wp);
    }
  }
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
