// sf_noalloc.cu -- sf_solve_static: a bounded solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside a host callback or
// a driver extension that must not allocate, a real-time loop that forbids
// allocation after start-up, a process whose memory pool is owned by another
// framework, or an embedding that only hands over pointers to its own buffers.
// For them this file provides one entry point whose workspace and tables live
// in a file-scope device array of fixed size.  Every GPU that loads the library
// holds that array (SF_STATIC_SCRATCH_BYTES) until the process exits.
//
// The solve itself is the same general engine as the plan-based path (the
// tile functions of sf_tiles.cuh, one launch per pass); only where its
// workspace comes from differs.  The pass descriptors travel as kernel
// arguments, and the twiddle / phase / eigenvalue tables are computed by a
// small kernel into the array, so nothing is uploaded from host memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/sailfish_gb300.h"
#include "sf_kernels.cuh"

using namespace sfg;

#define SF_STATIC_SCRATCH_BYTES (64u << 20)  // 64 MiB, shared by every call on a device
#define SF_STATIC_MAX_DEVICES 64

// The array itself.  Host code must never pass its name to a kernel (in host
// code it is only a stand-in for the symbol); the device address is obtained
// with cudaGetSymbolAddress once per CUDA context on each device.
static __device__ __align__(256) unsigned char sf_static_scratch[SF_STATIC_SCRATCH_BYTES];

namespace sfg {
void set_last_error_text(const std::string &msg);  // the text sf_last_error returns (sf_api.cu)
}

namespace {

sf_status na_fail(sf_status s, const std::string &msg) {
  set_last_error_text("sf_solve_static: " + msg);
  return s;
}

#define NA_CK(call)                                                                                       \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return na_fail(SF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__global__ void __launch_bounds__(SF_THREADS) k_static_pass(Prob<float> prob, Pass<float> pass);

// Device address of the array in the CUDA context current on each device.  An
// address belongs to one context: after cudaDeviceReset (or in another
// driver-API context on the same device) the module is loaded again and the
// array may sit elsewhere.  Each entry is therefore keyed by the context's
// unique ID (cuCtxGetId, reached through the runtime's driver entry-point
// query, so the library does not link the driver directly); a call in a new
// context repeats the set-up: the symbol lookup and the kernel's shared-memory
// attribute.
struct StaticState {
  unsigned long long ctx_id;
  unsigned char *addr;
};
StaticState g_state[SF_STATIC_MAX_DEVICES] = {};
std::mutex g_state_mu;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// unique ID of the current context; false when it cannot be read
bool current_ctx_id(unsigned long long *id) {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PfnCtxGetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(p);
  });
  if (!get_cur || !get_id) return false;
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

sf_status scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  NA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= SF_STATIC_MAX_DEVICES) return na_fail(SF_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lk(g_state_mu);
  StaticState &st = g_state[dev];
  unsigned long long id = 0;
  const bool have_id = st.addr && current_ctx_id(&id);
  if (!have_id || id != st.ctx_id) {
    // set-up in this context (the lookup also initialises the context when needed)
    void *p = nullptr;
    NA_CK(cudaGetSymbolAddress(&p, sf_static_scratch));
    NA_CK(cudaFuncSetAttribute(k_static_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, SF_SMEM_BUDGET));
    st.addr = static_cast<unsigned char *>(p);
    // without a readable context ID the address is looked up on every call
    st.ctx_id = current_ctx_id(&id) ? id : 0;
    if (!st.ctx_id) {
      *out = st.addr;
      st.addr = nullptr;
      return SF_OK;
    }
  }
  *out = st.addr;
  return SF_OK;
}

// one pass, descriptors by value (copied to shared memory like the plan path)
__global__ void __launch_bounds__(SF_THREADS) k_static_pass(Prob<float> prob, Pass<float> pass) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(16) Prob<float> sP;
  __shared__ Pass<float> sPass;
  if (threadIdx.x == 0) {
    sP = prob;
    sPass = pass;
  }
  __syncthreads();
  run_tile<float>(sP, sPass, blockIdx.x, reinterpret_cast<cx<float> *>(sm), (size_t)sPass.bufsz);
}

// tables of one axis in FP64 (CUDA's sincospi), rounded to float:
// twiddles exp(-2 pi i j / L), phases of the DST/DCT extensions, Table 1
// eigenvalues per coefficient index (PS or FD2)
__global__ void k_static_tables(float2 *tw, float2 *phase, float *lam, float *kap, float *kap2, int kind, int n, int L,
                                int ns, int k0, int eig, double Ldom) {
  const double h = Ldom / n;
  const double pi = 3.14159265358979323846264338327950288;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * j / L, &s, &c);
    tw[j] = make_float2((float)c, (float)s);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
    double s, c, re = 1.0, im = 0.0;
    sincospi(k / (2.0 * n), &s, &c);
    if (kind == AK_DR) { re = 0.0; im = -1.0; }
    else if (kind == AK_NS) { re = c; im = s; }
    else if (kind == AK_DS) { re = s; im = -c; }
    phase[k] = make_float2((float)re, (float)im);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
    double v;
    if (kind == AK_P) {
      const int kk = min(i, n - i);
      if (eig == SF_EIG_PS) v = -(2.0 * pi * kk / Ldom) * (2.0 * pi * kk / Ldom);
      else {
        const double sn = sinpi((double)i / n);
        v = -(4.0 / (h * h)) * sn * sn;
      }
    } else {
      const int m = i + k0;
      if (eig == SF_EIG_PS) v = -(pi * m / Ldom) * (pi * m / Ldom);
      else {
        const double sn = sinpi(m / (2.0 * n));
        v = -(4.0 / (h * h)) * sn * sn;
      }
    }
    lam[i] = (float)v;
    kap[i] = 0.f;
    kap2[i] = 0.f;
  }
}

int radix_plan_static(int L, int *rad) {
  int n = 0, m = L;
  if (m % 3 == 0) {
    rad[n++] = 3;
    m /= 3;
  }
  while (m >= 16) {
    rad[n++] = 16;
    m /= 16;
  }
  if (m > 1) rad[n++] = m;
  return n;
}

bool len_ok(int L) {
  if (L < 4 || L > 2048) return false;
  int m = L % 3 == 0 ? L / 3 : L;
  return (m & (m - 1)) == 0;
}

struct Carve {
  unsigned char *base;
  size_t used, cap;
  void *take(size_t bytes) {
    const size_t off = (used + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

}  // namespace

extern "C" sf_status sf_solve_static(const sf_plan_desc *d, const void *dev_f, void *dev_psi, void *cuda_stream) {
  if (!d || !dev_f || !dev_psi) return na_fail(SF_ERR_ARG, "null argument");
  if (d->prec != SF_F32) return na_fail(SF_ERR_UNSUPPORTED, "computes in FP32 only");
  if (d->dim != 2 && d->dim != 3) return na_fail(SF_ERR_ARG, "dim must be 2 or 3");
  if (d->ncomp != 1 || d->op != SF_OP_NONE) return na_fail(SF_ERR_UNSUPPORTED, "one component, no operator");
  if (d->grid != SF_GRID_REGULAR && d->grid != SF_GRID_STAGGERED) return na_fail(SF_ERR_ARG, "bad grid type");
  if (d->eig != SF_EIG_PS && d->eig != SF_EIG_FD2) return na_fail(SF_ERR_ARG, "bad eigenvalue type");
  if (!(d->rhs_scale == d->rhs_scale) || d->rhs_scale == 0.0 || std::isinf(d->rhs_scale))
    return na_fail(SF_ERR_ARG, "rhs_scale must be finite and non-zero");
  int nper = 0, nreal = 0;
  int kinds[3] = {AK_P, AK_P, AK_P};
  for (int a = 0; a < d->dim; ++a) {
    const int bc = d->bc[a][0];
    if (bc != d->bc[a][1]) return na_fail(SF_ERR_UNSUPPORTED, "different boundary types on one axis");
    if (bc == SF_BC_UNBOUNDED) return na_fail(SF_ERR_UNSUPPORTED, "periodic, Dirichlet or Neumann axes only");
    if (bc < SF_BC_PERIODIC || bc > SF_BC_NEUMANN) return na_fail(SF_ERR_ARG, "bad boundary type");
    if (!(d->hi[a] > d->lo[a])) return na_fail(SF_ERR_ARG, "domain bounds need hi > lo");
    const bool stag = d->grid == SF_GRID_STAGGERED;
    kinds[a] = bc == SF_BC_PERIODIC ? AK_P : (bc == SF_BC_DIRICHLET ? (stag ? AK_DS : AK_DR) : (stag ? AK_NS : AK_NR));
    const int minn = kinds[a] == AK_DR ? 3 : 2;
    if (d->n[a] < minn) return na_fail(SF_ERR_ARG, "too few cells on an axis");
    if (d->n[a] > 2048) return na_fail(SF_ERR_UNSUPPORTED, "more than 2048 cells on an axis");
    const int L = kinds[a] == AK_P ? d->n[a] : 2 * d->n[a];
    if (!len_ok(L)) return na_fail(SF_ERR_UNSUPPORTED, "FFT length " + std::to_string(L) + " is not 2^p or 3*2^p in [4, 2048]");
    if (bc == SF_BC_PERIODIC) ++nper;
    else ++nreal;
  }
  if (nper && nreal) return na_fail(SF_ERR_UNSUPPORTED, "mixing periodic with Dirichlet/Neumann axes");
  if (nper && d->n[0] % 2) return na_fail(SF_ERR_UNSUPPORTED, "odd periodic x length");

  // ---- problem geometry (the same rules as plan creation) ----
  Prob<float> P{};
  P.dim = d->dim;
  P.ncomp = P.nin = P.nout = 1;
  P.cpath = nper ? 1 : 0;
  P.rhs_scale = (float)d->rhs_scale;
  double prodL = 1.0;
  int L_[3] = {1, 1, 1};
  for (int a = 0; a < 3; ++a) {
    Axis<float> &x = P.ax[a];
    if (a >= d->dim) {
      x.kind = AK_P;
      x.n = x.nodes = x.nu = x.L = x.ns = 1;
      continue;
    }
    const int n = d->n[a];
    x.kind = kinds[a];
    x.n = n;
    switch (x.kind) {
      case AK_P: x.nodes = n; x.u0 = 0; x.nu = n; x.L = n; x.k0 = 0; break;
      case AK_DR: x.nodes = n + 1; x.u0 = 1; x.nu = n - 1; x.L = 2 * n; x.k0 = 1; break;
      case AK_NR: x.nodes = n + 1; x.u0 = 0; x.nu = n + 1; x.L = 2 * n; x.k0 = 0; break;
      case AK_DS: x.nodes = n; x.u0 = 0; x.nu = n; x.L = 2 * n; x.k0 = 1; break;
      default: x.nodes = n; x.u0 = 0; x.nu = n; x.L = 2 * n; x.k0 = 0; break;  // AK_NS
    }
    x.ns = P.cpath ? (a == 0 ? x.L / 2 + 1 : x.L) : x.nu;
    x.nst = radix_plan_static(x.L, x.radix);
    L_[a] = x.L;
    prodL *= x.L;
  }
  P.mscale = (float)(d->rhs_scale / prodL);
  P.nsx = P.ax[0].ns;
  P.nuy = P.ax[1].nu;
  P.nsy = P.ax[1].ns;
  P.nuz = d->dim == 3 ? P.ax[2].nu : 1;
  P.nsz = d->dim == 3 ? P.ax[2].ns : 1;
  {
    const int ndx = P.ax[0].nodes, ndy = P.ax[1].nodes, ndz = d->dim == 3 ? P.ax[2].nodes : 1;
    int fill = 0;
    if (P.ax[1].kind == AK_DR) fill += 2 * ndz * ndx;
    if (d->dim == 3 && P.ax[2].kind == AK_DR) fill += 2 * ndy * ndx;
    P.fill_count = fill;
  }

  // ---- carve tables and workspace out of the static array (size check first) ----
  const size_t esz = P.cpath ? sizeof(float2) : sizeof(float);
  const size_t eA = (size_t)P.nsx * P.nuz * P.nuy;
  const size_t eI = d->dim == 3 ? (size_t)P.nsx * P.nuz * P.nsy : 0;
  size_t need = 0;
  for (int a = 0; a < d->dim; ++a)
    need += 5 * 256 + (size_t)L_[a] * 8 + (size_t)(P.ax[a].n + 1) * 8 + 3 * (size_t)P.ax[a].ns * 4;
  need += 4 * 256 + 2 * eA * esz + 2 * eI * esz;
  if (need > SF_STATIC_SCRATCH_BYTES)
    return na_fail(SF_ERR_ARG, "problem needs " + std::to_string(need) + " bytes of workspace; sf_solve_static holds " +
                                   std::to_string((size_t)SF_STATIC_SCRATCH_BYTES) + " (use sf_plan_create)");

  unsigned char *scratch = nullptr;
  {
    const sf_status s = scratch_for_current_device(&scratch);
    if (s != SF_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Carve cv{scratch, 0, SF_STATIC_SCRATCH_BYTES};
  for (int a = 0; a < d->dim; ++a) {
    Axis<float> &x = P.ax[a];
    float2 *tw = (float2 *)cv.take((size_t)x.L * 8);
    float2 *ph = (float2 *)cv.take((size_t)(x.n + 1) * 8);
    float *lam = (float *)cv.take((size_t)x.ns * 4);
    float *kap = (float *)cv.take((size_t)x.ns * 4);
    float *kap2 = (float *)cv.take((size_t)x.ns * 4);
    if (!tw || !ph || !lam || !kap || !kap2) return na_fail(SF_ERR_ARG, "workspace does not fit the static array");
    k_static_tables<<<8, 256, 0, st>>>(tw, ph, lam, kap, kap2, x.kind, x.n, x.L, x.ns, x.k0, d->eig,
                                       d->hi[a] - d->lo[a]);
    NA_CK(cudaGetLastError());
    x.tw = tw;
    x.phase = ph;
    x.lam = lam;
    x.kap = kap;
    x.kap2 = kap2;
  }
  P.A = cv.take(eA * esz);
  P.B = cv.take(eA * esz);
  if (eI) {
    P.I1 = cv.take(eI * esz);
    P.I2 = cv.take(eI * esz);
  }
  if (!P.A || !P.B || (eI && (!P.I1 || !P.I2))) return na_fail(SF_ERR_ARG, "workspace does not fit the static array");
  P.in_ptr[0] = (const float *)dev_f;
  P.out_ptr[0] = (float *)dev_psi;
  // nothing in the array has to start at zero: every pass writes all the
  // workspace entries that a later pass reads, and the tables are rewritten

  // ---- passes (x, y[, z] forward with the multiply in the last stage, inverse) ----
  static_assert(sizeof(Pass<float>) < 256, "pass descriptor travels as a kernel argument");
  auto launch = [&](int kind, int L, int nbuf, int lines) -> sf_status {
    Pass<float> ps{};
    ps.kind = kind;
    ps.dep[0] = ps.dep[1] = -1;
    int W = 16;
    while (W > 1 && W / 2 >= lines) W >>= 1;
    for (;; W >>= 1) {
      const int Wp = W > 1 ? W + 1 : 1;
      const size_t bs = std::max((size_t)L * Wp, (size_t)(L + 2) * W);
      if (W == 1 || nbuf * bs * sizeof(float2) <= SF_SMEM_BUDGET) {
        ps.W = W;
        ps.Wp = Wp;
        ps.nbuf = nbuf;
        ps.bufsz = (int)bs;
        break;
      }
    }
    const int RPT = lines_per_tile(P.cpath, ps.W);
    switch (kind) {
      case PK_XFWD: ps.ntiles = P.nuz * cdiv(P.nuy, 2 * ps.W); break;
      case PK_YFWD: ps.ntiles = P.nsx * cdiv(P.nuz, RPT); break;
      case PK_ZSTAGE: ps.ntiles = P.nsx * cdiv(P.nsy, RPT); break;
      case PK_YINV: ps.ntiles = P.nsx * cdiv(P.nuz, RPT); break;
      case PK_XINV: ps.ntiles = P.nuz * cdiv(P.nuy, 2 * ps.W); break;
      case PK_YSTAGE2: ps.ntiles = cdiv(P.nsx, RPT); break;
      default: ps.ntiles = cdiv(P.fill_count, 4096); ps.W = ps.Wp = 1; ps.nbuf = 0; ps.bufsz = 0; break;
    }
    if (ps.ntiles <= 0) return SF_OK;
    const size_t smem = (size_t)ps.nbuf * ps.bufsz * sizeof(float2);
    k_static_pass<<<ps.ntiles, SF_THREADS, smem, st>>>(P, ps);
    NA_CK(cudaGetLastError());
    return SF_OK;
  };
  sf_status s;
  if ((s = launch(PK_XFWD, P.ax[0].L, 2, cdiv(P.nuy, 2))) != SF_OK) return s;
  if (d->dim == 3) {
    const int rows = P.cpath ? P.nuz : cdiv(P.nuz, 2);
    if ((s = launch(PK_YFWD, P.ax[1].L, 2, rows)) != SF_OK) return s;
    if ((s = launch(PK_ZSTAGE, P.ax[2].L, 3, P.cpath ? P.nsy : cdiv(P.nsy, 2))) != SF_OK) return s;
    if ((s = launch(PK_YINV, P.ax[1].L, 2, rows)) != SF_OK) return s;
  } else {
    if ((s = launch(PK_YSTAGE2, P.ax[1].L, 3, P.cpath ? P.nsx : cdiv(P.nsx, 2))) != SF_OK) return s;
  }
  if ((s = launch(PK_XINV, P.ax[0].L, 2, cdiv(P.nuy, 2))) != SF_OK) return s;
  if (P.fill_count && (s = launch(PK_FILL, 1, 0, 1)) != SF_OK) return s;
  return SF_OK;
}
