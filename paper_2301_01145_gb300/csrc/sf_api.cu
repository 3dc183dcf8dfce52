// sf_api.cu -- host implementation of the C ABI declared in include/sailfish_gb300.h.
//
// Plan creation follows the initialisation sequence of Sec. 2.4.4 (grid
// set-up, transform plans, Green's function or eigenvalues, operators); the
// solve follows the execution sequence of Sec. 2.4.5.  All tables are built
// in FP64 (host libm for twiddles, phases, eigenvalues and wavenumbers; FP64
// GPU kernels for the Green's function and its transform) and rounded once
// to the plan's precision.
#include <cuda_runtime.h>

#include <atomic>

#include <nvtx3/nvToolsExt.h>  // header-only NVTX v3: named ranges for profilers, a no-op without one

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sailfish_gb300.h"
#include "sf_engine.cuh"
#include "sf_fast.cuh"

using namespace sfg;

namespace {

thread_local std::string g_err;

sf_status fail(sf_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

}  // namespace

// the text sf_last_error returns, set by entry points in other files
namespace sfg {
void set_last_error_text(const std::string &msg) { g_err = msg; }
}  // namespace sfg

namespace {

#define SF_CK(call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(SF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define SF_TRY(expr)              \
  do {                            \
    sf_status s_ = (expr);        \
    if (s_ != SF_OK) return s_;   \
  } while (0)

const double kPi = 3.14159265358979323846264338327950288;
const size_t kSmemBudget = SF_SMEM_BUDGET;
const int kMaxW = 16;
const unsigned long long kTimeoutNs = 2000000000ull;  // 2 s bound on any scheduler wait

bool valid_len(int L) {
  if (L < 4 || L > 2048) return false;
  int m = L;
  if (m % 3 == 0) m /= 3;
  return (m & (m - 1)) == 0;
}

// radix plan: one radix-3 stage if needed, then stages of the largest radix
// allowed (16 by default), then the remainder (2, 4 or 8)
int radix_plan(int L, int *rad, int maxr) {
  if (maxr != 2 && maxr != 4 && maxr != 8) maxr = 16;
  int n = 0;
  int m = L;
  if (m % 3 == 0) {
    rad[n++] = 3;
    m /= 3;
  }
  while (m >= maxr) {
    rad[n++] = maxr;
    m /= maxr;
  }
  if (m > 1) rad[n++] = m;
  return n;
}

struct AxisHost {
  int kind, n, nodes, u0, nu, L, ns, k0, nst, radix[5];
  double Ldom, h;
  std::vector<double> tw, twf, phase, lam, kap, kap2;  // complex tables interleaved re,im
};

// per-axis transform geometry and tables (Table 1; Sec. 2.4.3 wavenumbers)
// smallest FFT length of the form 2^p or 3 * 2^p (>= 4) that is at least m
static int pad_length(int m) {
  m = std::max(m, 4);
  int best = 0;
  for (int base : {1, 3}) {
    int v = base;
    while (v < m) v *= 2;
    if (!best || v < best) best = v;
  }
  return best;
}

// regular: an unbounded axis on the regular grid (N_c + 1 nodes, padded to pad_length(2 N_c + 1))
AxisHost build_axis(int kind, int n, double lo, double hi, int eig, bool is_x, bool cpath, int maxr = 16,
                    bool regular = false) {
  AxisHost a{};
  a.kind = kind;
  a.n = n;
  a.Ldom = hi - lo;
  a.h = a.Ldom / n;
  switch (kind) {
    case AK_P: a.nodes = n; a.u0 = 0; a.nu = n; a.L = n; a.k0 = 0; break;
    case AK_U:
      a.nodes = regular ? n + 1 : n;
      a.u0 = 0;
      a.nu = a.nodes;
      a.L = regular ? pad_length(2 * n + 1) : 2 * n;
      a.k0 = 0;
      break;
    case AK_DR: a.nodes = n + 1; a.u0 = 1; a.nu = n - 1; a.L = 2 * n; a.k0 = 1; break;
    case AK_NR: a.nodes = n + 1; a.u0 = 0; a.nu = n + 1; a.L = 2 * n; a.k0 = 0; break;
    case AK_DS: a.nodes = n; a.u0 = 0; a.nu = n; a.L = 2 * n; a.k0 = 1; break;
    case AK_NS: a.nodes = n; a.u0 = 0; a.nu = n; a.L = 2 * n; a.k0 = 0; break;
    // one Dirichlet and one Neumann face: the Dirichlet axis of 2n cells, mirrored
    case AK_DNR: a.nodes = n + 1; a.u0 = 1; a.nu = n; a.L = 4 * n; a.k0 = 1; break;
    case AK_NDR: a.nodes = n + 1; a.u0 = 0; a.nu = n; a.L = 4 * n; a.k0 = 1; break;
    case AK_DNS: a.nodes = n; a.u0 = 0; a.nu = n; a.L = 4 * n; a.k0 = 1; break;
    case AK_NDS: a.nodes = n; a.u0 = 0; a.nu = n; a.L = 4 * n; a.k0 = 1; break;
  }
  if (cpath) a.ns = is_x ? a.L / 2 + 1 : a.L;
  else a.ns = a.nu;
  a.nst = radix_plan(a.L, a.radix, maxr);
  const int L = a.L;
  a.tw.resize(2 * (size_t)L);
  for (int j = 0; j < L; ++j) {
    const double ang = -2.0 * kPi * (double)j / (double)L;
    a.tw[2 * j] = std::cos(ang);
    a.tw[2 * j + 1] = std::sin(ang);
  }
  // warp-FFT twiddles (L = 32 E): [k1][t] = W_L^{t k1} (k1 < E, t < 32), then
  // [j][q] = W_L^{q j E} (j < E, q < G = 32 / E), then [mm - 1 + r] = W_{2 mm}^r
  // for the lane stages mm = 2, 4, .. < G (r < mm)
  if (L == 256 || L == 512) {
    const int E = L / 32, G = 32 / E;
    std::vector<double> ang;
    for (int k1 = 0; k1 < E; ++k1)
      for (int t = 0; t < 32; ++t) ang.push_back(-2.0 * kPi * (double)(t * k1) / L);
    for (int j = 0; j < E; ++j)
      for (int q = 0; q < G; ++q) ang.push_back(-2.0 * kPi * (double)(q * j * E) / L);
    for (int mm = 1; mm < G; mm <<= 1)
      for (int r = 0; r < mm; ++r) ang.push_back(-2.0 * kPi * (double)r / (2.0 * mm));
    if (L == 512) {
      // parity-split stages (sf_par.cuh): W_512^{u (2 k1 + p)} as [p][k1][u], then as [p][u][k1]
      ang.resize(SF_TWP_OFF, 0.0);
      for (int tr = 0; tr < 2; ++tr)
        for (int p = 0; p < 2; ++p)
          for (int i = 0; i < 16; ++i)
            for (int j = 0; j < 16; ++j) {
              const int k1 = tr ? j : i, u = tr ? i : j;
              ang.push_back(-2.0 * kPi * (double)(u * (2 * k1 + p)) / 512.0);
            }
    }
    a.twf.resize(2 * ang.size());
    for (size_t i = 0; i < ang.size(); ++i) {
      a.twf[2 * i] = std::cos(ang[i]);
      a.twf[2 * i + 1] = std::sin(ang[i]);
    }
  }
  // phases over k in [0, L/2]; a mixed axis takes those of its doubled Dirichlet axis
  const int half = L / 2;
  const int pkind = (kind == AK_DNR || kind == AK_NDR) ? AK_DR : ((kind == AK_DNS || kind == AK_NDS) ? AK_DS : kind);
  a.phase.assign(2 * (size_t)(half + 1), 0.0);
  for (int k = 0; k <= half; ++k) {
    double re = 1, im = 0;
    const double c = std::cos(kPi * k / (2.0 * half)), s = std::sin(kPi * k / (2.0 * half));
    switch (pkind) {
      case AK_DR: re = 0; im = -1; break;
      case AK_NS: re = c; im = s; break;
      case AK_DS: re = s; im = -c; break;  // -i e^{i pi k/2n}
      default: break;
    }
    a.phase[2 * k] = re;
    a.phase[2 * k + 1] = im;
  }
  a.lam.assign(a.ns, 0.0);
  a.kap.assign(a.ns, 0.0);
  a.kap2.assign(a.ns, 0.0);
  for (int i = 0; i < a.ns; ++i) {
    if (kind == AK_P) {
      const int k = i;  // FFT index (x: half spectrum)
      const int kk = std::min(k, n - k);
      if (eig == SF_EIG_PS) a.lam[i] = -std::pow(2.0 * kPi * kk / a.Ldom, 2);
      else a.lam[i] = -(4.0 / (a.h * a.h)) * std::pow(std::sin(kPi * k / n), 2);
    } else if (ak_mixed(kind)) {
      const double m = i + 0.5;  // quarter-wave mode k + 1/2 (odd mode 2k+1 of the doubled axis)
      if (eig == SF_EIG_PS) a.lam[i] = -std::pow(kPi * m / a.Ldom, 2);
      else a.lam[i] = -(4.0 / (a.h * a.h)) * std::pow(std::sin(kPi * m / (2.0 * n)), 2);
    } else if (kind != AK_U) {
      const int m = i + a.k0;  // mode number of Table 1
      if (eig == SF_EIG_PS) a.lam[i] = -std::pow(kPi * m / a.Ldom, 2);
      else a.lam[i] = -(4.0 / (a.h * a.h)) * std::pow(std::sin(kPi * m / (2.0 * n)), 2);
    }
    if (cpath) {
      const int M = L;  // points of the periodic (possibly doubled) axis
      const double period = (kind == AK_U) ? L * a.h : a.Ldom;  // the padded axis for unbounded
      const int k = i;
      int ks = (k <= M / 2) ? k : k - M;
      const double kap2v = std::pow(2.0 * kPi * std::min(k, M - k) / period, 2);
      if (M % 2 == 0 && k == M / 2) ks = 0;  // Nyquist: no odd derivative
      a.kap[i] = 2.0 * kPi * ks / period;
      a.kap2[i] = kap2v;
    }
  }
  return a;
}

// allocation failure injection (sf_debug_fail_alloc): remaining successes, < 0 = off
static std::atomic<long long> g_alloc_budget{-1};

#define SF_GUARD_BYTES 4096
#define SF_GUARD_BYTE 0xA5

template <typename T> struct DevMem {
  std::vector<void *> ptrs;
  bool guarded = false;  // SF_FLAG_DEBUG_CHECKS: guard bands around every allocation
  std::vector<std::pair<unsigned char *, size_t>> guards;  // (start, bytes) of each band
  ~DevMem() {
    for (void *p : ptrs) cudaFree(p);
  }
  sf_status alloc(void **out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) return SF_OK;
    long long b = g_alloc_budget.load();
    while (b >= 0) {
      if (b == 0) return fail(SF_ERR_OOM, "device allocation refused by the failure injection hook");
      if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    const size_t pad = guarded ? SF_GUARD_BYTES : 0;
    const size_t body = (bytes + 255) / 256 * 256;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, body + 2 * pad);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA,
                  std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    ptrs.push_back(base);
    unsigned char *b8 = static_cast<unsigned char *>(base);
    if (pad) {
      SF_CK(cudaMemset(b8, SF_GUARD_BYTE, pad));
      SF_CK(cudaMemset(b8 + pad + body, SF_GUARD_BYTE, pad));
      guards.push_back({b8, pad});
      guards.push_back({b8 + pad + body, pad});
    }
    *out = b8 + pad;
    return SF_OK;
  }
  template <typename U> sf_status upload(U **out, const std::vector<double> &v, bool complex_pairs) {
    std::vector<U> tmp(v.size());
    for (size_t i = 0; i < v.size(); ++i) tmp[i] = (U)v[i];
    void *p = nullptr;
    SF_TRY(alloc(&p, tmp.size() * sizeof(U)));
    if (!tmp.empty()) SF_CK(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(U), cudaMemcpyHostToDevice));
    *out = (U *)p;
    (void)complex_pairs;
    return SF_OK;
  }
};

template <typename T> sf_status fill_axis(Axis<T> &d, const AxisHost &h, DevMem<T> &mem) {
  d.kind = h.kind;
  d.n = h.n;
  d.nodes = h.nodes;
  d.u0 = h.u0;
  d.nu = h.nu;
  d.L = h.L;
  d.ns = h.ns;
  d.k0 = h.k0;
  d.nst = h.nst;
  for (int i = 0; i < 5; ++i) d.radix[i] = h.radix[i];
  T *tw, *twf, *ph, *lam, *kap, *kap2;
  SF_TRY(mem.template upload<T>(&tw, h.tw, true));
  SF_TRY(mem.template upload<T>(&twf, h.twf, true));
  SF_TRY(mem.template upload<T>(&ph, h.phase, true));
  SF_TRY(mem.template upload<T>(&lam, h.lam, false));
  SF_TRY(mem.template upload<T>(&kap, h.kap, false));
  SF_TRY(mem.template upload<T>(&kap2, h.kap2, false));
  d.tw = reinterpret_cast<const cx<T> *>(tw);
  d.twf = reinterpret_cast<const cx<T> *>(twf);
  d.phase = reinterpret_cast<const cx<T> *>(ph);
  d.lam = lam;
  d.kap = kap;
  d.kap2 = kap2;
  return SF_OK;
}

// ---------------------------------------------------------------------------
// pass lists and their execution
// ---------------------------------------------------------------------------
template <typename T> int pass_tiles(const Prob<T> &P, const Pass<T> &ps) {
  const int W = ps.W;
  switch (ps.kind) {
    case PK_XFWD: return P.nin * P.nuz * cdiv(P.nuy, 2 * W);
    case PK_YFWD: return P.nin * P.nsx * cdiv(P.nuz, lines_per_tile(P.cpath, W));
    case PK_ZSTAGE: return P.nsx * cdiv(P.nsy, lines_per_tile(P.cpath, W));
    case PK_YINV: return P.nout * P.nsx * cdiv(P.nuz, lines_per_tile(P.cpath, W));
    case PK_XINV: return P.nout * P.nuz * cdiv(P.nuy, 2 * W);
    case PK_YSTAGE2: return cdiv(P.nsx, lines_per_tile(P.cpath, W));
    case PK_FILL: return cdiv(P.fill_count * P.nout, 4096);
    case PK_ZFWD: return P.nsx * cdiv(P.nsy, 2 * W);
    case PK_MULT1D: return cdiv(P.nsx, SF_MULT1D_MODES);
    case PK_DERIV: {
      const int a = ps.arg[0];
      const int nlines = P.ax[a == 0 ? 1 : 0].nodes * P.ax[a == 2 ? 1 : 2].nodes;
      return cdiv(nlines, 2 * W);
    }
    case PK_DXINV:  // every (y, z) node line
      return (P.dim == 3 ? P.ax[2].nodes : 1) * cdiv(P.dim >= 2 ? P.ax[1].nodes : 1, 2 * W);
    case PK_YTERM:  // every z node row of every kx
      return P.nsx * cdiv(P.ax[2].nodes, 2 * W);
  }
  return 0;
}

// choose the tile width W (packed lines) for a pass: largest power of two that
// fits the shared-memory budget and does not exceed the lines available
template <typename T> void size_pass(const Prob<T> &P, Pass<T> &ps, int wcap) {
  int L = 0, nbuf = 2, lines = 1;
  switch (ps.kind) {
    case PK_XFWD: L = P.ax[0].L; lines = cdiv(P.nuy, 2); break;
    case PK_XINV: L = P.ax[0].L; lines = cdiv(P.nuy, 2); break;
    case PK_DXINV: L = P.ax[0].L; lines = cdiv(P.dim >= 2 ? P.ax[1].nodes : 1, 2); break;
    case PK_YTERM: L = P.ax[1].L; lines = cdiv(P.ax[2].nodes, 2); break;
    case PK_YFWD:
    case PK_YINV: L = P.ax[1].L; lines = P.cpath ? P.nuz : cdiv(P.nuz, 2); break;
    case PK_ZSTAGE: L = P.ax[2].L; nbuf = P.ncomp + 2; lines = P.cpath ? P.nsy : cdiv(P.nsy, 2); break;
    case PK_YSTAGE2: L = P.ax[1].L; nbuf = P.ncomp + 2; lines = P.cpath ? P.nsx : cdiv(P.nsx, 2); break;
    case PK_ZFWD: L = P.ax[2].L; lines = cdiv(P.nsy, 2); break;
    case PK_DERIV: {
      const int a = ps.arg[0];
      L = P.ax[a].L;
      lines = cdiv(P.ax[a == 0 ? 1 : 0].nodes * P.ax[a == 2 ? 1 : 2].nodes, 2);
      break;
    }
    case PK_FILL:
    case PK_MULT1D: ps.W = 1; ps.Wp = 1; ps.nbuf = 0; ps.bufsz = 0; return;
  }
  int W = kMaxW;
  if (wcap >= 1 && wcap < kMaxW)
    while (W > wcap) W >>= 1;
  while (W > 1 && W / 2 >= lines) W >>= 1;
  for (;; W >>= 1) {
    const int Wp = W > 1 ? W + 1 : 1;
    const size_t bs = std::max((size_t)L * Wp, (size_t)(L + 2) * W);
    if (W == 1 || nbuf * bs * sizeof(cx<T>) <= kSmemBudget) {
      ps.W = W;
      ps.Wp = Wp;
      ps.nbuf = nbuf;
      ps.bufsz = (int)bs;
      return;
    }
  }
}

template <typename T> struct ExecList {
  std::vector<Pass<T>> passes;
  std::vector<int> start;
  Pass<T> *d_passes = nullptr;
  int *d_start = nullptr;
  unsigned *d_done = nullptr;
  size_t smem = 0;
  int total = 0;
  int wcap = 0;  // tile-width cap (tuning)

  void add(const Prob<T> &P, int kind, int prob, int dep0 = -1, int dep1 = -1, const int *args = nullptr) {
    Pass<T> ps{};
    ps.kind = kind;
    ps.prob = prob;
    if (args)
      for (int i = 0; i < 6; ++i) ps.arg[i] = args[i];
    size_pass<T>(P, ps, wcap);
    ps.ntiles = pass_tiles<T>(P, ps);
    ps.dep[0] = dep0;
    ps.dep[1] = dep1;
    ps.depcnt[0] = dep0 >= 0 ? passes[dep0].ntiles : 0;
    ps.depcnt[1] = dep1 >= 0 ? passes[dep1].ntiles : 0;
    if (ps.ntiles > 0) passes.push_back(ps);
  }
  sf_status upload(DevMem<T> &mem) {
    start.assign(passes.size() + 1, 0);
    smem = 0;
    for (size_t i = 0; i < passes.size(); ++i) {
      start[i + 1] = start[i] + passes[i].ntiles;
      smem = std::max(smem, (size_t)passes[i].nbuf * passes[i].bufsz * sizeof(cx<T>));
    }
    total = start.back();
    void *p;
    SF_TRY(mem.alloc(&p, std::max<size_t>(1, passes.size()) * sizeof(Pass<T>)));
    d_passes = (Pass<T> *)p;
    SF_TRY(mem.alloc(&p, start.size() * sizeof(int)));
    d_start = (int *)p;
    SF_TRY(mem.alloc(&p, std::max<size_t>(1, passes.size()) * sizeof(unsigned)));
    d_done = (unsigned *)p;
    if (!passes.empty()) SF_CK(cudaMemcpy(d_passes, passes.data(), passes.size() * sizeof(Pass<T>), cudaMemcpyHostToDevice));
    SF_CK(cudaMemcpy(d_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
    return SF_OK;
  }
};

// kernel attributes are per device: set them once on each device that launches
template <typename T> sf_status set_kernel_attrs() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  SF_CK(cudaGetDevice(&dev));
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load() & bit)) return SF_OK;
  SF_CK(engine_set_attrs<T>());
  done.fetch_or(bit);
  return SF_OK;
}

// add the dependency edges of a linear chain: each pass waits for all tiles of
// the previous one (FILL touches disjoint nodes and waits for nothing)
template <typename T>
sf_status launch_list(ExecList<T> &ex, const Prob<T> *d_probs, bool fused, cudaStream_t st, ExecCtl *ctl, unsigned *sticky,
                      const IOArgs<T> &io, int *launches) {
  SF_TRY(set_kernel_attrs<T>());
  if (ex.passes.empty()) return SF_OK;
  if (fused) {
    SF_CK(cudaMemsetAsync(ex.d_done, 0, ex.passes.size() * sizeof(unsigned), st));
    SF_CK(cudaMemsetAsync(ctl, 0, sizeof(ExecCtl), st));
    int dev = 0, nsm = 0, per = 0;
    SF_CK(cudaGetDevice(&dev));
    SF_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SF_CK(engine_exec_occupancy<T>(&per, ex.smem));
    if (per < 1) return fail(SF_ERR_CUDA, "executor does not fit on an SM");
    const int grid = std::min(ex.total, nsm * per);
    SF_CK(engine_launch_exec<T>(grid, ex.smem, st, d_probs, ex.d_passes, ex.d_start, (int)ex.passes.size(), ex.d_done,
                                ctl, sticky, kTimeoutNs, io));
    if (launches) *launches += 1;
  } else {
    for (size_t i = 0; i < ex.passes.size(); ++i) {
      const Pass<T> &ps = ex.passes[i];
      const size_t sm = (size_t)ps.nbuf * ps.bufsz * sizeof(cx<T>);
      SF_CK(engine_launch_pass<T>(ps.ntiles, sm, st, d_probs, ex.d_passes, (int)i, io));
      if (launches) *launches += 1;
    }
  }
  return SF_OK;
}


// ---------------------------------------------------------------------------
// fast path (register warp FFT) for equal-length periodic/unbounded 3D FP32 solves
// ---------------------------------------------------------------------------
struct FastList {
  std::vector<FPass> passes;
  std::vector<int> start;
  FPass *d_passes = nullptr;
  int *d_start = nullptr;
  unsigned *d_done = nullptr;
  int total = 0;
};

// slab pipeline with stage lag D: step t issues YF(t), ZS(t-D), YI(t-2D).  The
// I1 / I2 rings have nslot = D + 2 slabs: a slot is rewritten only after the
// pass that reads it (dependency edges below), and with one slot beyond the D + 1
// in flight that pass was issued a full step (all three passes) earlier, so the
// wait is normally already satisfied.  Every dependency points to an earlier
// item of the list.  Unfused plans (nslot = 1) launch the passes one by one.
template <typename T>
void build_fast_list(const Prob<T> &Q, int S, int nslot, int L, FastList &fl) {
  const int nslab = cdiv(Q.nsx, S);
  const int D = nslot > 2 ? nslot - 2 : 1;
  std::vector<int> iyf(nslab, -1), izs(nslab, -1), iyi(nslab, -1);
  auto push = [&](int kind, int s) {
    FPass p{};
    p.kind = kind;
    p.kx0 = s * S;
    p.nkx = std::min(S, Q.nsx - s * S);
    p.slot = s % nslot;
    p.dep[0] = p.dep[1] = -1;
    if (kind == FK_YF) {
      p.ntiles = fast_tiles_yf(Q, p.nkx);
      if (s >= nslot) p.dep[0] = izs[s - nslot];
    } else if (kind == FK_ZS) {
      p.ntiles = fast_tiles_zs(p.nkx, L) * (fast_split_curl(Q) ? 3 : 1);
      p.dep[0] = iyf[s];
      if (s >= nslot) p.dep[1] = iyi[s - nslot];
    } else {
      p.ntiles = fast_tiles_yi(Q, p.nkx);
      p.dep[0] = izs[s];
    }
    for (int d = 0; d < 2; ++d) p.depcnt[d] = p.dep[d] >= 0 ? fl.passes[p.dep[d]].ntiles : 0;
    fl.passes.push_back(p);
    const int idx = (int)fl.passes.size() - 1;
    if (kind == FK_YF) iyf[s] = idx;
    else if (kind == FK_ZS) izs[s] = idx;
    else iyi[s] = idx;
  };
  for (int step = 0; step < nslab + 2 * D; ++step) {
    if (step < nslab) push(FK_YF, step);
    if (step - D >= 0 && step - D < nslab) push(FK_ZS, step - D);
    if (step - 2 * D >= 0 && step - 2 * D < nslab) push(FK_YI, step - 2 * D);
  }
  fl.start.assign(fl.passes.size() + 1, 0);
  for (size_t i = 0; i < fl.passes.size(); ++i) fl.start[i + 1] = fl.start[i] + fl.passes[i].ntiles;
  fl.total = fl.start.back();
}

template <typename T> sf_status upload_fast(FastList &fl, DevMem<T> &mem) {
  void *p;
  SF_TRY(mem.alloc(&p, fl.passes.size() * sizeof(FPass)));
  fl.d_passes = (FPass *)p;
  SF_TRY(mem.alloc(&p, fl.start.size() * sizeof(int)));
  fl.d_start = (int *)p;
  SF_TRY(mem.alloc(&p, fl.passes.size() * sizeof(unsigned)));
  fl.d_done = (unsigned *)p;
  SF_CK(cudaMemcpy(fl.d_passes, fl.passes.data(), fl.passes.size() * sizeof(FPass), cudaMemcpyHostToDevice));
  SF_CK(cudaMemcpy(fl.d_start, fl.start.data(), fl.start.size() * sizeof(int), cudaMemcpyHostToDevice));
  return SF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// the plan object
// ---------------------------------------------------------------------------
// CUDA-event marks around the kernels of full solves: one event before the
// first kernel, between consecutive kernels and after the last; a ring keeps
// the marks of the last kRing solves.
struct KernelTimer {
  static const int kRing = 256, kMarks = 4;
  bool on = false;
  long long count = 0;
  int nmark = 0;  // marks of the last recorded solve (slots = nmark - 1)
  std::vector<cudaEvent_t> ev;
  ~KernelTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  sf_status enable(bool en) {
    if (en && ev.empty()) {
      ev.resize(kRing * kMarks, nullptr);
      for (auto &e : ev) SF_CK(cudaEventCreate(&e));
    }
    on = en;
    count = 0;
    nmark = 0;
    return SF_OK;
  }
  // the marks of the next solve, or nullptr when timing is off or the stream is being captured
  cudaEvent_t *next(cudaStream_t st) {
    if (!on) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    return &ev[(size_t)(count % kRing) * kMarks];
  }
  void done(int marks) {
    nmark = marks;
    ++count;
  }
};

struct sf_plan_s {
  virtual ~sf_plan_s() {}
  sf_plan_desc d{};
  cudaStream_t stream = nullptr;
  bool is_batch = false;
  int launches_per_exec = 0;
  KernelTimer timer;
  virtual sf_status solve_part(bool front, bool back, const void *f, void *psi, void *op, int *launches) = 0;
  virtual sf_status adjoint(const void *gp, const void *go, void *gf) = 0;
  virtual sf_status sync() = 0;
  virtual sf_status query(size_t in_shape[4], size_t out_shape[4], size_t op_shape[4], size_t *ws) = 0;
  virtual sf_status set_face(int axis, int side, const void *p) = 0;
  virtual sf_status host_solve(const void *hf, void *hpsi, void *hop) = 0;
  virtual sf_status host_solve_many(int n, const void *const *hf, void *const *hpsi, void *const *hop) = 0;
  virtual sf_status corrupt_guard() { return fail(SF_ERR_STATE, "not available on a batch"); }
  virtual ExecCtl *exec_ctl() = 0;
  const void *src = nullptr;
  bool solved = false;
};

template <typename T> struct PlanImpl : sf_plan_s {
  DevMem<T> mem;
  Prob<T> P{};   // forward problem
  Prob<T> PA{};  // adjoint problem
  Prob<T> *d_probs = nullptr;  // [0] forward, [1] adjoint
  ExecList<T> ex_front, ex_back, ex_all, ex_adj;
  // first-derivative operators on Dirichlet / Neumann axes: the adjoint first
  // forms h = g_psi + D^T g_op (derivative passes, ex_adjop) and then runs the
  // transposed solve on h
  ExecList<T> ex_adjop;
  T *adj_h = nullptr;
  bool deriv_ops = false;
  ExecCtl *ctl = nullptr;
  unsigned *sticky = nullptr;
  const T *faces[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  size_t ws_bytes = 0;
  size_t field_elems = 0, op_elems = 0;
  int fastE = 0;  // 8 or 16: register fast path with L = 32 E; 0: generic engine
  bool semi = false;  // one unbounded axis, the others periodic
  FastGeo geo{};
  FastList fl_fwd, fl_adj;
  void *st_in = nullptr, *st_psi = nullptr, *st_op = nullptr;  // host-solve staging

  bool fused() const { return !(d.flags & SF_FLAG_UNFUSED); }

  IOArgs<T> io_forward(const void *f, void *psi, void *op) const {
    IOArgs<T> io{};
    io.use = 1;
    for (int c = 0; c < P.ncomp; ++c) io.in[c] = f ? (const T *)f + c * field_elems : nullptr;
    for (int c = 0; c < P.ncomp; ++c) io.out[c] = psi ? (T *)psi + c * field_elems : nullptr;
    for (int o = 0; o < P.nop; ++o) io.out[P.ncomp + o] = op ? (T *)op + o * field_elems : nullptr;
    int hf = 0;
    for (int a = 0; a < 3; ++a)
      for (int s = 0; s < 2; ++s) {
        io.face[a][s] = faces[a][s];
        if (faces[a][s]) hf = 1;
      }
    io.has_face = hf;
    return io;
  }

  sf_status init(const sf_plan_desc &desc, cudaStream_t st);
  sf_status build_green();
  sf_status build_green_semi(const AxisHost *ah);

  // on: the stream to launch on (the plan's stream when null)
  sf_status run_fast(const Prob<T> &Q, const Prob<T> *dq, FastList &fl, bool front, bool back, const IOArgs<T> &io,
                     int *launches, cudaEvent_t *marks = nullptr, cudaStream_t on = nullptr);

  sf_status solve_part(bool front, bool back, const void *f, void *psi, void *op, int *launches) override {
    IOArgs<T> io = io_forward(f, psi, op);
    cudaEvent_t *mk = front && back ? timer.next(stream) : nullptr;
    if (fastE) {
      SF_TRY(run_fast(P, d_probs, fl_fwd, front, back, io, launches, mk));
      if (mk) timer.done(4);
      return SF_OK;
    }
    if (front && back) {
      if (mk) SF_CK(cudaEventRecord(mk[0], stream));
      SF_TRY(launch_list<T>(ex_all, d_probs, fused(), stream, ctl, sticky, io, launches));
      if (mk) {
        SF_CK(cudaEventRecord(mk[1], stream));
        timer.done(2);
      }
      return SF_OK;
    }
    if (front) return launch_list<T>(ex_front, d_probs, fused(), stream, ctl, sticky, io, launches);
    return launch_list<T>(ex_back, d_probs, fused(), stream, ctl, sticky, io, launches);
  }

  sf_status adjoint(const void *gp, const void *go, void *gf) override {
    if (deriv_ops) {
      // h = g_psi + D^T g_op, then the transposed solve of h
      const size_t hb = (size_t)P.ncomp * field_elems * sizeof(T);
      if (gp) SF_CK(cudaMemcpyAsync(adj_h, gp, hb, cudaMemcpyDeviceToDevice, stream));
      else SF_CK(cudaMemsetAsync(adj_h, 0, hb, stream));
      if (go) {
        IOArgs<T> hio{};
        hio.use = 1;
        for (int o = 0; o < P.nop; ++o) hio.in[P.ncomp + o] = (const T *)go + o * field_elems;
        for (int c = 0; c < P.ncomp; ++c) hio.out[c] = adj_h + c * field_elems;
        hio.has_face = 0;
        SF_TRY(launch_list<T>(ex_adjop, d_probs, fused(), stream, ctl, sticky, hio, nullptr));
      }
      gp = adj_h;
      go = nullptr;
    }
    IOArgs<T> io{};
    io.use = 1;
    for (int c = 0; c < P.ncomp; ++c) io.in[c] = gp ? (const T *)gp + c * field_elems : nullptr;
    for (int o = 0; o < P.nop; ++o) io.in[P.ncomp + o] = go ? (const T *)go + o * field_elems : nullptr;
    for (int c = 0; c < P.ncomp; ++c) io.out[c] = (T *)gf + c * field_elems;
    io.has_face = 0;
    if (fastE) return run_fast(PA, d_probs + 1, fl_adj, true, true, io, nullptr);
    return launch_list<T>(ex_adj, d_probs + 1, fused(), stream, ctl, sticky, io, nullptr);
  }

  sf_status sync() override {
    SF_CK(cudaStreamSynchronize(stream));
    unsigned s = 0;
    SF_CK(cudaMemcpy(&s, sticky, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (s) {
      SF_CK(cudaMemset(sticky, 0, sizeof(unsigned)));
      return fail(SF_ERR_TIMEOUT, "a scheduler wait exceeded its bound; results are invalid");
    }
    return check_guards();
  }

  // SF_FLAG_DEBUG_CHECKS: every guard band must still hold SF_GUARD_BYTE
  sf_status check_guards() {
    if (!mem.guarded) return SF_OK;
    std::vector<unsigned char> h(SF_GUARD_BYTES);
    for (size_t i = 0; i < mem.guards.size(); ++i) {
      SF_CK(cudaMemcpy(h.data(), mem.guards[i].first, mem.guards[i].second, cudaMemcpyDeviceToHost));
      for (size_t j = 0; j < mem.guards[i].second; ++j)
        if (h[j] != SF_GUARD_BYTE)
          return fail(SF_ERR_CORRUPT, "guard band " + std::to_string(i) + " of the plan's workspace overwritten at byte " +
                                          std::to_string(j));
    }
    return SF_OK;
  }

  sf_status corrupt_guard() override {
    if (!mem.guarded || mem.guards.empty()) return fail(SF_ERR_STATE, "plan has no guard bands (SF_FLAG_DEBUG_CHECKS)");
    SF_CK(cudaStreamSynchronize(stream));
    SF_CK(cudaMemset(mem.guards[0].first + 7, 0x00, 1));
    return SF_OK;
  }

  sf_status query(size_t in_shape[4], size_t out_shape[4], size_t op_shape[4], size_t *ws) override {
    const size_t nz = d.dim == 3 ? P.ax[2].nodes : 1;
    const size_t s3[3] = {nz, (size_t)P.ax[1].nodes, (size_t)P.ax[0].nodes};
    if (in_shape) {
      in_shape[0] = P.ncomp;
      for (int i = 0; i < 3; ++i) in_shape[i + 1] = s3[i];
    }
    if (out_shape) {
      out_shape[0] = P.ncomp;
      for (int i = 0; i < 3; ++i) out_shape[i + 1] = s3[i];
    }
    if (op_shape) {
      op_shape[0] = P.nop;
      for (int i = 0; i < 3; ++i) op_shape[i + 1] = P.nop ? s3[i] : 0;
    }
    if (ws) *ws = ws_bytes;
    return SF_OK;
  }

  sf_status set_face(int axis, int side, const void *p) override {
    if (axis < 0 || axis >= d.dim || side < 0 || side > 1) return fail(SF_ERR_ARG, "axis/side out of range");
    const int k = P.ax[axis].kind;
    if (p && (k == AK_P || k == AK_U))
      return fail(SF_ERR_ARG, "boundary data needs a Dirichlet or Neumann axis");
    if (p && d.eig != SF_EIG_FD2) return fail(SF_ERR_UNSUPPORTED, "inhomogeneous boundaries need FD2 eigenvalues (Sec. 2.5.2)");
    if (p && P.ncomp != 1) return fail(SF_ERR_UNSUPPORTED, "boundary data only for scalar solves");
    faces[axis][side] = (const T *)p;
    return SF_OK;
  }

  ExecCtl *exec_ctl() override { return ctl; }

  sf_status host_solve(const void *hf, void *hpsi, void *hop) override {
    const size_t fb = field_elems * sizeof(T);
    if (!st_in) {
      SF_TRY(mem.alloc(&st_in, fb * P.ncomp));
      SF_TRY(mem.alloc(&st_psi, fb * P.ncomp));
      if (P.nop) SF_TRY(mem.alloc(&st_op, fb * P.nop));
    }
    SF_CK(cudaMemcpyAsync(st_in, hf, fb * P.ncomp, cudaMemcpyHostToDevice, stream));
    SF_TRY(solve_part(true, true, st_in, st_psi, st_op, nullptr));
    SF_CK(cudaMemcpyAsync(hpsi, st_psi, fb * P.ncomp, cudaMemcpyDeviceToHost, stream));
    if (P.nop && hop) SF_CK(cudaMemcpyAsync(hop, st_op, fb * P.nop, cudaMemcpyDeviceToHost, stream));
    return sync();
  }

  // n host solves in a pipeline: the upload of solve i+1 and the download of
  // solve i-1 run on two side streams while solve i runs on the plan stream;
  // NSTAGE device staging sets rotate, ordered by events, so that a solve
  // waits only for the download of the solve NSTAGE steps back
  static constexpr int NSTAGE = 3;
  void *pin[NSTAGE] = {}, *ppsi[NSTAGE] = {}, *pop[NSTAGE] = {};
  cudaStream_t s_up = nullptr, s_down = nullptr;
  cudaEvent_t ev_up[NSTAGE] = {}, ev_comp[NSTAGE] = {}, ev_down[NSTAGE] = {};

  ~PlanImpl() override {
    if (s_up) cudaStreamSynchronize(s_up);
    if (s_down) cudaStreamSynchronize(s_down);
    for (int b = 0; b < NSTAGE; ++b) {
      if (ev_up[b]) cudaEventDestroy(ev_up[b]);
      if (ev_comp[b]) cudaEventDestroy(ev_comp[b]);
      if (ev_down[b]) cudaEventDestroy(ev_down[b]);
    }
    if (s_up) cudaStreamDestroy(s_up);
    if (s_down) cudaStreamDestroy(s_down);
  }

  sf_status host_solve_many(int n, const void *const *hf, void *const *hpsi, void *const *hop) override {
    const size_t fb = field_elems * sizeof(T);
    if (!s_up) {
      for (int b = 0; b < NSTAGE; ++b) {
        SF_TRY(mem.alloc(&pin[b], fb * P.ncomp));
        SF_TRY(mem.alloc(&ppsi[b], fb * P.ncomp));
        if (P.nop) SF_TRY(mem.alloc(&pop[b], fb * P.nop));
        SF_CK(cudaEventCreateWithFlags(&ev_up[b], cudaEventDisableTiming));
        SF_CK(cudaEventCreateWithFlags(&ev_comp[b], cudaEventDisableTiming));
        SF_CK(cudaEventCreateWithFlags(&ev_down[b], cudaEventDisableTiming));
      }
      SF_CK(cudaStreamCreateWithFlags(&s_up, cudaStreamNonBlocking));
      SF_CK(cudaStreamCreateWithFlags(&s_down, cudaStreamNonBlocking));
    }
    for (int i = 0; i < n; ++i) {
      const int b = i % NSTAGE;
      if (i >= NSTAGE) SF_CK(cudaStreamWaitEvent(s_up, ev_comp[b], 0));  // the solve that read pin[b] is done
      SF_CK(cudaMemcpyAsync(pin[b], hf[i], fb * P.ncomp, cudaMemcpyHostToDevice, s_up));
      SF_CK(cudaEventRecord(ev_up[b], s_up));
      SF_CK(cudaStreamWaitEvent(stream, ev_up[b], 0));
      if (i >= NSTAGE) SF_CK(cudaStreamWaitEvent(stream, ev_down[b], 0));  // its outputs are home
      SF_TRY(solve_part(true, true, pin[b], ppsi[b], pop[b], nullptr));
      SF_CK(cudaEventRecord(ev_comp[b], stream));
      SF_CK(cudaStreamWaitEvent(s_down, ev_comp[b], 0));
      SF_CK(cudaMemcpyAsync(hpsi[i], ppsi[b], fb * P.ncomp, cudaMemcpyDeviceToHost, s_down));
      if (P.nop && hop && hop[i]) SF_CK(cudaMemcpyAsync(hop[i], pop[b], fb * P.nop, cudaMemcpyDeviceToHost, s_down));
      SF_CK(cudaEventRecord(ev_down[b], s_down));
    }
    SF_CK(cudaStreamSynchronize(s_up));
    SF_CK(cudaStreamSynchronize(s_down));
    return sync();
  }
};

template <typename T>
sf_status PlanImpl<T>::run_fast(const Prob<T> &, const Prob<T> *, FastList &, bool, bool, const IOArgs<T> &, int *,
                                cudaEvent_t *, cudaStream_t) {
  return fail(SF_ERR_UNSUPPORTED, "fast path is FP32 only");
}
template <>
sf_status PlanImpl<float>::run_fast(const Prob<float> &Q, const Prob<float> *dq, FastList &fl, bool front, bool back,
                                    const IOArgs<float> &io, int *launches, cudaEvent_t *marks, cudaStream_t on) {
  FastLaunch L{};
  L.marks = marks;
  L.d_prob = dq;
  L.h_prob = &Q;
  L.geo = geo;
  L.d_passes = fl.d_passes;
  L.d_start = fl.d_start;
  L.d_done = fl.d_done;
  L.npass = (int)fl.passes.size();
  L.total = fl.total;
  L.ctl = ctl;
  L.sticky = sticky;
  L.timeout_ns = kTimeoutNs;
  L.front = front;
  L.back = back;
  L.stream = on ? on : stream;
  const int e = fastE == 16 ? sf_fast_launch_e16(L, io, launches) : sf_fast_launch_e8(L, io, launches);
  if (e) return fail(SF_ERR_CUDA, std::string("fast path launch: ") + cudaGetErrorString((cudaError_t)e));
  return SF_OK;
}

static int axis_kind(int bc, int grid, int bc_hi = -1) {
  const bool stag = grid == SF_GRID_STAGGERED;
  if (bc_hi >= 0 && bc_hi != bc) {  // one Dirichlet and one Neumann face
    if (bc == SF_BC_DIRICHLET && bc_hi == SF_BC_NEUMANN) return stag ? AK_DNS : AK_DNR;
    if (bc == SF_BC_NEUMANN && bc_hi == SF_BC_DIRICHLET) return stag ? AK_NDS : AK_NDR;
    return -1;
  }
  switch (bc) {
    case SF_BC_PERIODIC: return AK_P;
    case SF_BC_UNBOUNDED: return AK_U;
    case SF_BC_DIRICHLET: return stag ? AK_DS : AK_DR;
    case SF_BC_NEUMANN: return stag ? AK_NS : AK_NR;
  }
  return -1;
}

static int op_outputs(int op, int dim, int ncomp) {
  switch (op) {
    case SF_OP_GRAD: return dim;
    case SF_OP_DIV: return 1;
    case SF_OP_CURL: return dim == 3 ? 3 : 2;
    case SF_OP_NABLA: return ncomp;
  }
  return 0;
}

static sf_status validate(const sf_plan_desc &d) {
  if (d.dim < 1 || d.dim > 3) return fail(SF_ERR_ARG, "dim must be 1, 2 or 3");
  if (d.flags & ~(SF_FLAG_UNFUSED | SF_FLAG_GENERIC | SF_FLAG_DEBUG_CHECKS)) return fail(SF_ERR_ARG, "unknown flag bits");
  if (d.prec != SF_F32 && d.prec != SF_F64) return fail(SF_ERR_ARG, "prec must be SF_F32 or SF_F64");
  if (d.grid != SF_GRID_REGULAR && d.grid != SF_GRID_STAGGERED) return fail(SF_ERR_ARG, "bad grid type");
  if (d.ncomp < 1 || d.ncomp > 3) return fail(SF_ERR_ARG, "ncomp must be 1..3");
  if (d.op < SF_OP_NONE || d.op > SF_OP_NABLA) return fail(SF_ERR_ARG, "bad operator");
  if (d.eig != SF_EIG_PS && d.eig != SF_EIG_FD2) return fail(SF_ERR_ARG, "bad eigenvalue type");
  if (!(d.rhs_scale == d.rhs_scale) || d.rhs_scale == 0.0 || std::isinf(d.rhs_scale))
    return fail(SF_ERR_ARG, "rhs_scale must be finite and non-zero");
  int ncp = 0, nreal = 0, nunb = 0;
  for (int a = 0; a < d.dim; ++a) {
    const int bc = d.bc[a][0];
    if (bc < SF_BC_PERIODIC || bc > SF_BC_UNBOUNDED) return fail(SF_ERR_ARG, "bad boundary type");
    if (d.bc[a][1] < SF_BC_PERIODIC || d.bc[a][1] > SF_BC_UNBOUNDED) return fail(SF_ERR_ARG, "bad boundary type");
    const bool mixed = d.bc[a][0] != d.bc[a][1];
    if (mixed && axis_kind(bc, d.grid, d.bc[a][1]) < 0)
      return fail(SF_ERR_UNSUPPORTED, "unequal faces on one axis: only a Dirichlet / Neumann pair is supported");
    if (!(d.hi[a] > d.lo[a]) || !std::isfinite(d.hi[a] - d.lo[a]))
      return fail(SF_ERR_ARG, "domain bounds need finite lo < hi");
    const int n = d.n[a];
    const int minn = (bc == SF_BC_DIRICHLET && d.grid == SF_GRID_REGULAR && !mixed) ? 3 : 2;
    if (n < minn) return fail(SF_ERR_ARG, "too few cells on an axis");
    if (n > 2048) return fail(SF_ERR_UNSUPPORTED, "more than 2048 cells on an axis");  // before any 2n / 4n
    const int L = bc == SF_BC_PERIODIC ? n
                  : mixed                  ? 4 * n
                  : (bc == SF_BC_UNBOUNDED && d.grid == SF_GRID_REGULAR) ? pad_length(2 * n + 1)
                                           : 2 * n;
    if (!valid_len(L)) return fail(SF_ERR_UNSUPPORTED, "FFT length " + std::to_string(L) + " is not 2^p or 3*2^p in [4, 2048]");
    if (bc == SF_BC_PERIODIC || bc == SF_BC_UNBOUNDED) ++ncp;
    else ++nreal;
    if (bc == SF_BC_UNBOUNDED) ++nunb;
  }
  if (ncp && nreal) return fail(SF_ERR_UNSUPPORTED, "mixing periodic/unbounded with Dirichlet/Neumann axes");
  const bool semi = nunb == 1 && d.dim >= 2 && ncp == d.dim;  // one unbounded axis, the others periodic
  if (nunb && nunb != d.dim && !semi)
    return fail(SF_ERR_UNSUPPORTED, "semi-unbounded domains need exactly one unbounded axis, the others periodic");
  if (nunb && !semi && (d.green < SF_GREEN_G2 || d.green > SF_GREEN_SPECTRAL)) return fail(SF_ERR_ARG, "bad kernel");
  if (nunb && d.dim == 1 && d.green != SF_GREEN_SPECTRAL)
    return fail(SF_ERR_UNSUPPORTED, "1D unbounded solves use the spectral kernel (SF_GREEN_SPECTRAL)");
  if (nunb && !semi && d.green != SF_GREEN_SPECTRAL && !(d.green_sigma > 0.0 && std::isfinite(d.green_sigma)))
    return fail(SF_ERR_ARG, "green_sigma must be positive and finite");
  if (ncp && d.bc[0][0] == SF_BC_PERIODIC && (d.n[0] % 2)) return fail(SF_ERR_UNSUPPORTED, "odd periodic x length");
  if (d.op != SF_OP_NONE) {
    if (d.op == SF_OP_GRAD && d.ncomp != 1) return fail(SF_ERR_ARG, "GRAD needs ncomp = 1");
    if (d.op == SF_OP_DIV && d.ncomp != d.dim) return fail(SF_ERR_ARG, "DIV needs ncomp = dim");
    if (d.op == SF_OP_CURL && d.dim == 1) return fail(SF_ERR_ARG, "CURL needs dim 2 or 3");
    if (d.op == SF_OP_CURL && d.ncomp != (d.dim == 3 ? 3 : 1)) return fail(SF_ERR_ARG, "CURL needs ncomp 3 (3D) or 1 (2D)");
  }
  if (d.ncomp + op_outputs(d.op, d.dim, d.ncomp) > SF_MAXF) return fail(SF_ERR_ARG, "too many fields");
  if (!(d.tune_radix == 0 || d.tune_radix == 2 || d.tune_radix == 4 || d.tune_radix == 8 || d.tune_radix == 16))
    return fail(SF_ERR_ARG, "tune_radix must be 0, 2, 4, 8 or 16");
  if (d.tune_tile < 0 || d.tune_tile > 16 || (d.tune_tile & (d.tune_tile - 1)))
    return fail(SF_ERR_ARG, "tune_tile must be 0 or a power of two up to 16");
  if (d.tune_slab < 0) return fail(SF_ERR_ARG, "tune_slab must be >= 0");
  if (d.tune_lag < 0 || d.tune_lag > 8) return fail(SF_ERR_ARG, "tune_lag must be in [0, 8]");
  return SF_OK;
}

template <typename T> static void derive_extents(Prob<T> &P) {
  P.nsx = P.ax[0].ns;
  P.nuy = P.ax[1].nu;
  P.nsy = P.ax[1].ns;
  P.nuz = P.dim == 3 ? P.ax[2].nu : 1;
  P.nsz = P.dim == 3 ? P.ax[2].ns : 1;
  const int ndx = P.ax[0].nodes, ndy = P.ax[1].nodes, ndz = P.dim == 3 ? P.ax[2].nodes : 1;
  int fill = 0;
  const int ym = dnode_mask(P.ax[1].kind), zm = P.dim == 3 ? dnode_mask(P.ax[2].kind) : 0;
  fill += ((ym & 1) + (ym >> 1)) * ndz * ndx;
  fill += ((zm & 1) + (zm >> 1)) * ndy * ndx;
  P.fill_count = fill;
}

template <typename T> sf_status PlanImpl<T>::init(const sf_plan_desc &desc, cudaStream_t st) {
  d = desc;
  stream = st;
  mem.guarded = (d.flags & SF_FLAG_DEBUG_CHECKS) != 0;
  SF_TRY(set_kernel_attrs<T>());
  Prob<T> &p = P;
  p.dim = d.dim;
  p.ncomp = d.ncomp;
  p.nop = op_outputs(d.op, d.dim, d.ncomp);
  p.op = d.op;
  const int k0 = axis_kind(d.bc[0][0], d.grid);
  p.cpath = (k0 == AK_P || k0 == AK_U) ? 1 : 0;
  int nunb = 0;
  for (int a = 0; a < d.dim; ++a) nunb += d.bc[a][0] == SF_BC_UNBOUNDED;
  semi = nunb > 0 && nunb < d.dim;  // validated: one unbounded axis, the others periodic
  p.green = nunb > 0 ? 1 : 0;
  p.rhs_scale = (T)d.rhs_scale;
  double prodL = 1.0, hd = 1.0;
  AxisHost ah[3];
  for (int a = 0; a < 3; ++a) {
    if (a < d.dim) {
      ah[a] = build_axis(axis_kind(d.bc[a][0], d.grid, d.bc[a][1]), d.n[a], d.lo[a], d.hi[a], d.eig, a == 0, p.cpath,
                         d.tune_radix, d.grid == SF_GRID_REGULAR);
      prodL *= ah[a].L;
      hd *= ah[a].h;
    } else {  // unused z axis of a 2D problem: a trivial periodic axis of one point
      ah[a] = AxisHost{};
      ah[a].kind = AK_P;
      ah[a].n = 1;
      ah[a].nodes = 1;
      ah[a].nu = 1;
      ah[a].L = 1;
      ah[a].ns = 1;
    }
    if (a < d.dim) SF_TRY(fill_axis<T>(p.ax[a], ah[a], mem));
    else {
      p.ax[a] = Axis<T>{};
      p.ax[a].kind = AK_P;
      p.ax[a].n = 1;
      p.ax[a].nodes = 1;
      p.ax[a].nu = 1;
      p.ax[a].L = 1;
      p.ax[a].ns = 1;
    }
  }
  p.mscale = (T)(d.rhs_scale / prodL);
  // operator coefficient table (Sec. 2.4.3): output o = sum_c coef(o, c) psi_c
  for (int o = 0; o < 3; ++o)
    for (int c = 0; c < 3; ++c) p.opc[o][c] = p.opa[o][c] = 0;
  auto deriv = [&](int o, int c, int sign, int axis) {
    p.opc[o][c] = sign;
    p.opa[o][c] = axis;
  };
  switch (d.op) {
    case SF_OP_GRAD:
      for (int a = 0; a < d.dim; ++a) deriv(a, 0, 1, a);
      break;
    case SF_OP_DIV:
      for (int a = 0; a < d.dim; ++a) deriv(0, a, 1, a);
      break;
    case SF_OP_CURL:
      if (d.dim == 3) {
        deriv(0, 2, 1, 1); deriv(0, 1, -1, 2);
        deriv(1, 0, 1, 2); deriv(1, 2, -1, 0);
        deriv(2, 1, 1, 0); deriv(2, 0, -1, 1);
      } else {
        deriv(0, 0, 1, 1); deriv(1, 0, -1, 0);
      }
      break;
    case SF_OP_NABLA:
      for (int c = 0; c < d.ncomp; ++c) p.opc[c][c] = 2;
      break;
  }
  derive_extents<T>(p);
  field_elems = (size_t)p.ax[0].nodes * p.ax[1].nodes * (d.dim == 3 ? p.ax[2].nodes : 1);
  // FD2 lifting weights (Sec. 2.5.2 boundary weighting; divided by rhs_scale
  // because the multiplier carries rhs_scale)
  for (int a = 0; a < d.dim; ++a) {
    const double h = ah[a].h;
    double w0 = 0, w1 = 0;
    if (ah[a].kind != AK_P && ah[a].kind != AK_U) {  // each face by its own type
      const bool reg = d.grid == SF_GRID_REGULAR;
      w0 = d.bc[a][0] == SF_BC_DIRICHLET ? (reg ? -1.0 : -2.0) / (h * h) : (reg ? 2.0 : 1.0) / h;
      w1 = d.bc[a][1] == SF_BC_DIRICHLET ? (reg ? -1.0 : -2.0) / (h * h) : -(reg ? 2.0 : 1.0) / h;
    }
    p.facew[a][0] = (T)(w0 / d.rhs_scale);
    p.facew[a][1] = (T)(w1 / d.rhs_scale);
  }
  // first-derivative terms of operators on Dirichlet / Neumann axes (reading
  // Z13), in the order the pass list takes them (outputs, then components): x
  // terms are formed from B, terms along the stage axis (y in 2D, z in 3D) in
  // the spectral stage, 3D y terms by the y-inverse term pass
  p.nst = p.n3yt = 0;
  if (!p.cpath && d.dim >= 2 && d.op != SF_OP_NONE && d.op != SF_OP_NABLA)
    for (int o = 0; o < p.nop; ++o)
      for (int c = 0; c < p.ncomp; ++c) {
        if (p.opc[o][c] != 1 && p.opc[o][c] != -1) continue;
        const int ax = p.opa[o][c];
        if (ax == d.dim - 1 && p.nst < SF_MAXYT) {
          p.st_comp[p.nst] = c;
          p.st_sgn[p.nst] = p.opc[o][c];
          ++p.nst;
        } else if (d.dim == 3 && ax == 1 && p.n3yt < SF_MAXYT) {
          p.yt_comp[p.n3yt] = c;
          p.yt_sgn[p.n3yt] = p.opc[o][c];
          ++p.n3yt;
        }
      }
  // workspace: every buffer sized for ncomp + nop fields (forward and adjoint)
  const int nf = p.ncomp + p.nop;
  const size_t esz = p.cpath ? sizeof(cx<T>) : sizeof(T);
  const size_t eA = (size_t)nf * p.nsx * p.nuz * p.nuy;
  size_t eI = d.dim == 3 ? (size_t)nf * p.nsx * p.nuz * p.nsy : 0;
  // register fast path: FP32, 3D, periodic/unbounded, one FFT length L = 256 or 512 on all axes
  if (sizeof(T) == 4 && d.dim == 3 && p.cpath && !semi && !(d.flags & SF_FLAG_GENERIC) && p.ax[0].L == p.ax[1].L &&
      p.ax[1].L == p.ax[2].L && (p.ax[0].L == 512 || p.ax[0].L == 256)) {
    fastE = p.ax[0].L / 32;
    int S = d.tune_slab > 0 ? d.tune_slab : 2;
    const int lag = d.tune_lag > 0 ? d.tune_lag : 1;
    geo.S = fused() ? std::min(S, p.nsx) : p.nsx;
    geo.nslot = fused() ? lag + 2 : 1;
    geo.nfmax = nf;
    eI = (size_t)geo.nslot * nf * geo.S * p.ax[1].L * p.nuz;
  }
  SF_TRY(mem.alloc(&p.A, eA * esz));
  // the derivative terms follow the psi fields, indexed by node: in B every
  // term as [t][kx][z node][y node], in I2 (3D) the z terms as [t][kx][z node][ky]
  const size_t ndy = d.dim >= 2 ? (size_t)p.ax[1].nodes : 1, ndz = d.dim == 3 ? (size_t)p.ax[2].nodes : 1;
  const size_t eB = std::max(eA, (size_t)p.ncomp * p.nsx * p.nuz * p.nuy + (size_t)(p.nst + p.n3yt) * p.nsx * ndz * ndy);
  const size_t eI2 = d.dim == 3 ? std::max(eI, (size_t)p.ncomp * p.nsx * p.nuz * p.nsy + (size_t)p.nst * p.nsx * ndz * p.nsy)
                                : eI;
  SF_TRY(mem.alloc(&p.B, eB * esz));
  if (eI) {
    SF_TRY(mem.alloc(&p.I1, eI * esz));
    SF_TRY(mem.alloc(&p.I2, eI2 * esz));
  }
  ws_bytes = (eA + eB + eI + eI2) * esz;
  void *tmp;
  SF_TRY(mem.alloc(&tmp, sizeof(ExecCtl)));
  ctl = (ExecCtl *)tmp;
  SF_TRY(mem.alloc(&tmp, sizeof(unsigned)));
  sticky = (unsigned *)tmp;
  SF_CK(cudaMemset(sticky, 0, sizeof(unsigned)));
  if (p.green && semi) {
    // table over the spectral indices: unbounded axis folded (L/2 + 1), periodic axes in full
    p.gny = ah[1].kind == AK_U ? ah[1].L / 2 + 1 : ah[1].L;
    p.gnz = d.dim == 3 ? (ah[2].kind == AK_U ? ah[2].L / 2 + 1 : ah[2].L) : 1;
    SF_TRY(build_green_semi(ah));
  } else if (p.green) {
    p.gny = ah[1].L / 2 + 1;  // octant of the padded axes
    p.gnz = d.dim == 3 ? ah[2].L / 2 + 1 : 1;
    SF_TRY(build_green());
    (void)hd;
  }
  // operators on Dirichlet / Neumann axes: dual bases (sine <-> cosine) and
  // wavenumber units; the operator outputs are then derivative passes over psi
  // (PK_DERIV) instead of spectral-stage outputs
  for (int a = 0; a < 3; ++a) {
    p.dkind[a] = p.ax[a].kind;
    p.du0[a] = p.ax[a].u0;
    p.dnu[a] = p.ax[a].nu;
    p.dk0[a] = p.ax[a].k0;
    p.dns[a] = p.ax[a].ns;
    p.dphase[a] = p.ax[a].phase;
    p.kunit[a] = 0;
    if (a >= d.dim || p.cpath || d.op == SF_OP_NONE) continue;
    static const int dual_of[10] = {AK_P, AK_U, AK_NR, AK_DR, AK_NS, AK_DS, AK_NDR, AK_NDS, AK_DNR, AK_DNS};
    const int dk = dual_of[p.ax[a].kind];
    AxisHost dh = build_axis(dk, d.n[a], d.lo[a], d.hi[a], d.eig, a == 0, false, d.tune_radix, d.grid == SF_GRID_REGULAR);
    T *dph;
    SF_TRY(mem.template upload<T>(&dph, dh.phase, true));
    p.dkind[a] = dk;
    p.du0[a] = dh.u0;
    p.dnu[a] = dh.nu;
    p.dk0[a] = dh.k0;
    p.dns[a] = dh.ns;
    p.dphase[a] = reinterpret_cast<const cx<T> *>(dph);
    p.kunit[a] = (T)(2.0 * kPi / (ah[a].L * ah[a].h));
  }
  // forward / adjoint variants
  p.nin = p.ncomp;
  p.nout = (p.cpath || d.op == SF_OP_NABLA) ? nf : p.ncomp;
  p.adjoint = 0;
  p.nrw = 0;
  PA = p;
  deriv_ops = !p.cpath && d.op != SF_OP_NONE && d.op != SF_OP_NABLA;
  PA.nin = deriv_ops ? p.ncomp : nf;  // derivative operators: their gradients enter through h
  PA.nout = p.ncomp;
  PA.adjoint = 1;
  PA.nst = PA.n3yt = 0;
  for (int a = 0; a < d.dim; ++a)
    if (p.ax[a].kind == AK_NR || p.ax[a].kind == AK_DNR || p.ax[a].kind == AK_NDR) PA.nrw = 1;
  SF_TRY(mem.alloc(&tmp, 2 * sizeof(Prob<T>)));
  d_probs = (Prob<T> *)tmp;
  SF_CK(cudaMemcpy(d_probs, &P, sizeof(Prob<T>), cudaMemcpyHostToDevice));
  SF_CK(cudaMemcpy(d_probs + 1, &PA, sizeof(Prob<T>), cudaMemcpyHostToDevice));
  // pass lists (Sec. 2.3 order: x, y, z forward; z, y, x inverse)
  auto front = [&](ExecList<T> &ex, const Prob<T> &Q) {
    ex.add(Q, PK_XFWD, 0);
    if (d.dim == 3) {
      ex.add(Q, PK_YFWD, 0, (int)ex.passes.size() - 1);
      ex.add(Q, PK_ZSTAGE, 0, (int)ex.passes.size() - 1);
      ex.add(Q, PK_YINV, 0, (int)ex.passes.size() - 1);
    } else if (d.dim == 2) {
      ex.add(Q, PK_YSTAGE2, 0, (int)ex.passes.size() - 1);
    } else {
      ex.add(Q, PK_MULT1D, 0, (int)ex.passes.size() - 1);
    }
  };
  auto back = [&](ExecList<T> &ex, const Prob<T> &Q, int dep) {
    ex.add(Q, PK_XINV, 0, dep);
    const int xinv = (int)ex.passes.size() - 1;
    if (Q.fill_count) ex.add(Q, PK_FILL, 0);
    if (Q.cpath || Q.op == OPK_NONE || Q.op == OPK_NABLA || Q.adjoint) return;
    // operator outputs on Dirichlet / Neumann axes: derivative terms, the
    // terms of one output chained (the first writes, the others add).  An x
    // derivative is formed from B, where x is still spectral (PK_DXINV); a y
    // or z derivative is a pass over the computed psi (PK_DERIV)
    int ist = 0, iyt = 0;  // stage terms and 3D y terms, in the order of the tables
    for (int o = 0; o < Q.nop; ++o) {
      int prev = -1;
      auto term = [&](int ax, int c, int order, int sign) {
        const int acc = prev >= 0 ? 1 : 0;
        int tb = -1;  // the term's index in B
        if (ax == Q.dim - 1 && ist < Q.nst) tb = ist++;
        else if (Q.dim == 3 && ax == 1 && iyt < Q.n3yt) tb = Q.nst + iyt++;
        if (ax == 0) {
          const int args[6] = {0, c, o, order, sign, acc};
          ex.add(Q, PK_DXINV, 0, dep, prev, args);
        } else if (tb >= 0) {
          int src = dep;  // 2D: the y stage wrote the term to B
          if (Q.dim == 3) {
            const int yargs[6] = {ax, tb, o, 0, 0, 0};
            ex.add(Q, PK_YTERM, 0, dep, -1, yargs);
            src = (int)ex.passes.size() - 1;
          }
          const int args[6] = {ax, tb, o, 4, sign, acc};
          ex.add(Q, PK_DXINV, 0, src, prev, args);
        } else {
          const int args[6] = {ax, c, o, order, sign, acc};
          ex.add(Q, PK_DERIV, 0, xinv, prev, args);
        }
        prev = (int)ex.passes.size() - 1;
      };
      for (int c = 0; c < Q.ncomp; ++c)
        if (Q.opc[o][c] == 1 || Q.opc[o][c] == -1) term(Q.opa[o][c], c, 1, Q.opc[o][c]);
    }
  };
  ex_front.wcap = ex_back.wcap = ex_all.wcap = ex_adj.wcap = d.tune_tile;
  front(ex_front, P);
  back(ex_back, P, -1);
  front(ex_all, P);
  back(ex_all, P, (int)ex_all.passes.size() - 1);
  {
    ExecList<T> &ex = ex_adj;
    front(ex, PA);
    back(ex, PA, (int)ex.passes.size() - 1);
    for (auto &ps : ex.passes) ps.prob = 0;  // d_probs + 1 is passed for the adjoint
  }
  if (deriv_ops) {
    // transposed derivative terms, all accumulating into h (chained)
    ex_adjop.wcap = d.tune_tile;
    int prev = -1;
    for (int o = 0; o < p.nop; ++o)
      for (int c = 0; c < p.ncomp; ++c)
        if (p.opc[o][c] == 1 || p.opc[o][c] == -1) {
          const int args[6] = {p.opa[o][c], c, o, 3, p.opc[o][c], 1};
          ex_adjop.add(p, PK_DERIV, 0, prev, -1, args);
          prev = (int)ex_adjop.passes.size() - 1;
        }
    SF_TRY(ex_adjop.upload(mem));
    void *hb;
    SF_TRY(mem.alloc(&hb, (size_t)p.ncomp * field_elems * sizeof(T)));
    adj_h = (T *)hb;
  }
  SF_TRY(ex_front.upload(mem));
  SF_TRY(ex_back.upload(mem));
  SF_TRY(ex_all.upload(mem));
  SF_TRY(ex_adj.upload(mem));
  launches_per_exec = fused() ? 1 : (int)ex_all.passes.size();
  if (fastE) {
    build_fast_list<T>(P, geo.S, geo.nslot, p.ax[1].L, fl_fwd);
    build_fast_list<T>(PA, geo.S, geo.nslot, p.ax[1].L, fl_adj);
    // the executor packs the pass table into shared memory (see k_fyz)
    if (fl_fwd.passes.size() > SF_FAST_MAXPASS || fl_adj.passes.size() > SF_FAST_MAXPASS)
      return fail(SF_ERR_UNSUPPORTED, "too many slab passes for the register path; raise tune_slab");
    SF_TRY(upload_fast<T>(fl_fwd, mem));
    SF_TRY(upload_fast<T>(fl_adj, mem));
    launches_per_exec = 3;
  }
  return SF_OK;
}

// Green's table (Sec. 2.6.2): G tabulated on the octant of the doubled grid in
// FP64, transformed by a 3D (2D) DCT-I -- the DFT of the mirrored table -- with
// the FP64 kernels, scaled by -rhs_scale h^d / prod(L) and rounded to T.
template <typename T> sf_status PlanImpl<T>::build_green() {
  const int dim = d.dim;
  // octant of the padded grid: L/2 + 1 offsets per axis (L = 2 N_c on staggered grids)
  const int nx = P.ax[0].L / 2, ny = P.ax[1].L / 2, nz = dim == 3 ? P.ax[2].L / 2 : 0;
  double h[3] = {0, 0, 0};
  double hd = 1.0, prodL = 1.0;
  for (int a = 0; a < dim; ++a) {
    h[a] = (d.hi[a] - d.lo[a]) / d.n[a];
    hd *= h[a];
    prodL *= (double)P.ax[a].L;
  }
  const size_t cnt = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  DevMem<double> tmem;
  void *oct, *A, *I1, *out;
  SF_TRY(tmem.alloc(&oct, cnt * sizeof(double)));
  SF_TRY(tmem.alloc(&A, cnt * sizeof(double)));
  SF_TRY(tmem.alloc(&I1, cnt * sizeof(double)));
  SF_TRY(tmem.alloc(&out, cnt * sizeof(double)));
  // Gaussian kernels: their order P; spectral kernel: order 0 with the cut-off pi / max h
  const int korder = d.green == SF_GREEN_SPECTRAL ? 0 : 2 * (d.green - SF_GREEN_G2) + 2;
  const double kc = kPi / std::max(h[0], std::max(h[1], dim == 3 ? h[2] : 0.0));
  sfg::k_green_octant<<<1024, 256, 0, stream>>>((double *)oct, nx, ny, nz, h[0], h[1], h[2], d.green_sigma, dim,
                                                 korder, kc);
  SF_CK(cudaGetLastError());
  // FP64 real-path problem: regular-Neumann (DCT-I) on every axis, forward only
  Prob<double> G{};
  G.dim = dim;
  G.ncomp = 1;
  G.nin = 1;
  G.nout = 1;
  G.cpath = 0;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      AxisHost ah = build_axis(AK_NR, P.ax[a].L / 2, 0.0, 1.0, SF_EIG_PS, a == 0, false);
      SF_TRY(fill_axis<double>(G.ax[a], ah, tmem));
    } else {
      G.ax[a] = Axis<double>{};
      G.ax[a].kind = AK_P;
      G.ax[a].n = G.ax[a].nodes = G.ax[a].nu = G.ax[a].L = G.ax[a].ns = 1;
    }
  }
  derive_extents<double>(G);
  G.A = A;
  G.I1 = dim == 3 ? I1 : out;
  G.fwd_out = (double *)out;
  void *dprob;
  SF_TRY(tmem.alloc(&dprob, sizeof(Prob<double>)));
  SF_CK(cudaMemcpy(dprob, &G, sizeof(Prob<double>), cudaMemcpyHostToDevice));
  ExecList<double> ex;
  ex.add(G, PK_XFWD, 0);
  if (dim >= 2) ex.add(G, PK_YFWD, 0, 0);
  if (dim == 3) ex.add(G, PK_ZFWD, 0, 1);
  SF_TRY(ex.upload(tmem));
  IOArgs<double> io{};
  io.use = 1;
  io.in[0] = (const double *)oct;
  SF_TRY(launch_list<double>(ex, (const Prob<double> *)dprob, false, stream, nullptr, nullptr, io, nullptr));
  void *gh;
  SF_TRY(mem.alloc(&gh, cnt * sizeof(T)));
  const double scale = -d.rhs_scale * hd / prodL;
  // 1D: the x transform's output (A) is the table
  sfg::k_convert_scale<T><<<1024, 256, 0, stream>>>((T *)gh, (const double *)(dim == 1 ? A : out), cnt, scale);
  SF_CK(cudaGetLastError());
  if (fastE && dim == 3) {
    void *ght;
    SF_TRY(mem.alloc(&ght, cnt * sizeof(T)));
    sfg::k_transpose_green<T><<<1024, 256, 0, stream>>>((T *)ght, (const T *)gh, nx + 1, nz + 1, ny + 1);
    SF_CK(cudaGetLastError());
    P.ghat_t = (const T *)ght;
  }
  SF_CK(cudaStreamSynchronize(stream));
  P.ghat = (const T *)gh;
  return SF_OK;
}

// Semi-unbounded Green's table (one unbounded axis ua, the others periodic):
// for every periodic mode, kappa^2 = -(sum of the periodic axes' Table 1
// eigenvalues, FP64 on the host), and along ua the DCT-I (the DFT of the
// mirrored row) of the free-space kernel of -(d^2/dz^2 - kappa^2) sampled on the
// doubled axis, exp(-kappa |z|) / (2 kappa) or -|z| / 2 for kappa = 0, scaled by
// -rhs_scale h_ua / prod(L) (FP64 kernel, then rounded to T).
template <typename T> sf_status PlanImpl<T>::build_green_semi(const AxisHost *ah) {
  const int dim = d.dim;
  int ua = 0;
  for (int a = 0; a < dim; ++a)
    if (ah[a].kind == AK_U) ua = a;
  const int ext[3] = {P.nsx, P.gny, dim == 3 ? P.gnz : 1};
  int pa = -1, pb = -1;  // the periodic axes, in increasing order
  for (int a = 0; a < dim; ++a)
    if (a != ua) (pa < 0 ? pa : pb) = a;
  const int ea = ext[pa], eb = pb >= 0 ? ext[pb] : 1;
  const size_t rows = (size_t)ea * eb;
  std::vector<double> kap2(rows);
  for (int i = 0; i < ea; ++i)
    for (int j = 0; j < eb; ++j)
      kap2[(size_t)i * eb + j] = -(ah[pa].lam[i] + (pb >= 0 ? ah[pb].lam[j] : 0.0));
  double prodL = 1.0;
  for (int a = 0; a < dim; ++a) prodL *= (double)P.ax[a].L;
  const size_t cnt = (size_t)ext[0] * ext[1] * ext[2];
  DevMem<double> tmem;
  void *dk, *out;
  SF_TRY(tmem.alloc(&dk, rows * sizeof(double)));
  SF_TRY(tmem.alloc(&out, cnt * sizeof(double)));
  SF_CK(cudaMemcpy(dk, kap2.data(), rows * sizeof(double), cudaMemcpyHostToDevice));
  const int Lu = P.ax[ua].L;
  const size_t smem = (size_t)(Lu + Lu / 2 + 1) * sizeof(double);
  SF_CK(cudaFuncSetAttribute(sfg::k_green_semi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sfg::k_green_semi<<<(unsigned)rows, 256, smem, stream>>>((double *)out, (const double *)dk, dim, ua, pa, pb, ext[0],
                                                            ext[1], ext[2], eb, Lu, ah[ua].h);
  SF_CK(cudaGetLastError());
  void *gh;
  SF_TRY(mem.alloc(&gh, cnt * sizeof(T)));
  sfg::k_convert_scale<T><<<1024, 256, 0, stream>>>((T *)gh, (const double *)out, cnt, -d.rhs_scale * ah[ua].h / prodL);
  SF_CK(cudaGetLastError());
  SF_CK(cudaStreamSynchronize(stream));
  P.ghat = (const T *)gh;
  return SF_OK;
}

// ---------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------
template <typename T> struct BatchImpl : sf_plan_s {
  DevMem<T> mem;
  std::vector<PlanImpl<T> *> plans;
  std::vector<Prob<T>> probs;
  Prob<T> *d_probs = nullptr;
  ExecList<T> ex;
  ExecCtl *ctl = nullptr;
  unsigned *sticky = nullptr;
  std::vector<const void *> last_f;
  std::vector<void *> last_psi, last_op;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture (the legacy stream cannot be captured)
  // members on the register fast path: their own launches (x forward, y/z
  // executor, x inverse) in the same graph, after the general members'
  // persistent launch; their buffers are kernel arguments, so a change of
  // buffers re-captures the graph
  std::vector<int> fastm;
  bool fast_ready = false;  // the fast members' kernels have run once outside a capture

  ~BatchImpl() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap) cudaStreamDestroy(cap);
  }

  sf_status init(const sf_plan *ps, int n, cudaStream_t st) {
    stream = st;
    is_batch = true;
    for (int i = 0; i < n; ++i) plans.push_back(static_cast<PlanImpl<T> *>(ps[i]));
    probs.resize(n);
    for (int i = 0; i < n; ++i) {
      probs[i] = plans[i]->P;
      if (plans[i]->fastE) fastm.push_back(i);
    }
    // level-synchronous order: every problem's pass j before any pass j+1, so a
    // problem's dependency is (almost always) complete when its next pass starts
    std::vector<std::vector<Pass<T>>> lists(n);
    for (int i = 0; i < n; ++i)
      if (!plans[i]->fastE) lists[i] = plans[i]->ex_all.passes;
    std::vector<int> last(n, -1);
    ex.wcap = plans[0]->d.tune_tile;
    size_t maxlen = 0;
    for (auto &k : lists) maxlen = std::max(maxlen, k.size());
    for (size_t lvl = 0; lvl < maxlen; ++lvl) {
      for (int i = 0; i < n; ++i) {
        if (lvl >= lists[i].size()) continue;
        const int kind = lists[i][lvl].kind;
        const int dep = (kind == PK_FILL) ? -1 : last[i];
        const size_t before = ex.passes.size();
        ex.add(probs[i], kind, i, dep, -1, lists[i][lvl].arg);
        if (ex.passes.size() > before && kind != PK_FILL) last[i] = (int)ex.passes.size() - 1;
      }
    }
    void *tmp;
    SF_TRY(mem.alloc(&tmp, std::max(1, n) * sizeof(Prob<T>)));
    d_probs = (Prob<T> *)tmp;
    SF_TRY(mem.alloc(&tmp, sizeof(ExecCtl)));
    ctl = (ExecCtl *)tmp;
    SF_TRY(mem.alloc(&tmp, sizeof(unsigned)));
    sticky = (unsigned *)tmp;
    SF_CK(cudaMemset(sticky, 0, sizeof(unsigned)));
    SF_TRY(ex.upload(mem));
    last_f.assign(n, nullptr);
    last_psi.assign(n, nullptr);
    last_op.assign(n, nullptr);
    launches_per_exec = (ex.passes.empty() ? 0 : 1) + 3 * (int)fastm.size();
    return SF_OK;
  }

  sf_status run(const void *const *f, void *const *psi, void *const *op) {
    const int n = (int)plans.size();
    for (int i = 0; i < n; ++i) {
      if (!f[i] || !psi[i]) return fail(SF_ERR_ARG, "null buffer in table");
      if (plans[i]->d.op != SF_OP_NONE && (!op || !op[i]))
        return fail(SF_ERR_ARG, "a plan with an operator needs its op output");
    }
    bool changed = !gexec;
    for (int i = 0; i < n; ++i) {
      void *o = op ? op[i] : nullptr;
      if (f[i] != last_f[i] || psi[i] != last_psi[i] || o != last_op[i]) changed = true;
    }
    if (changed) {
      SF_CK(cudaStreamSynchronize(stream));
      for (int i = 0; i < n; ++i) {
        Prob<T> &q = probs[i];
        PlanImpl<T> *pl = plans[i];
        void *o = op ? op[i] : nullptr;
        for (int c = 0; c < SF_MAXF; ++c) {
          q.in_ptr[c] = nullptr;
          q.out_ptr[c] = nullptr;
        }
        for (int c = 0; c < q.ncomp; ++c) {
          q.in_ptr[c] = (const T *)f[i] + c * pl->field_elems;
          q.out_ptr[c] = (T *)psi[i] + c * pl->field_elems;
        }
        for (int c = 0; c < q.nop; ++c) q.out_ptr[q.ncomp + c] = o ? (T *)o + c * pl->field_elems : nullptr;
        last_f[i] = f[i];
        last_psi[i] = psi[i];
        last_op[i] = o;
      }
      SF_CK(cudaMemcpy(d_probs, probs.data(), n * sizeof(Prob<T>), cudaMemcpyHostToDevice));
      if (gexec && !fastm.empty()) {
        SF_CK(cudaGraphExecDestroy(gexec));
        gexec = nullptr;
      }
      if (!fast_ready && !fastm.empty()) {
        // one uncaptured run sets the fast kernels' attributes (a solve into the given buffers)
        for (int i : fastm) {
          PlanImpl<T> *pl = plans[i];
          SF_TRY(pl->run_fast(pl->P, pl->d_probs, pl->fl_fwd, true, true, pl->io_forward(f[i], psi[i], op ? op[i] : nullptr),
                              nullptr, nullptr, stream));
        }
        SF_CK(cudaStreamSynchronize(stream));
        fast_ready = true;
      }
      if (!gexec) {
        // capture memsets + the persistent launch into a graph (Sec. "persistent batched scheduler")
        cudaGraph_t g;
        if (!cap) SF_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        SF_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        IOArgs<T> io{};
        io.use = 0;
        sf_status s = launch_list<T>(ex, d_probs, true, cap, ctl, sticky, io, nullptr);
        for (size_t m = 0; s == SF_OK && m < fastm.size(); ++m) {
          PlanImpl<T> *pl = plans[fastm[m]];
          const int i = fastm[m];
          s = pl->run_fast(pl->P, pl->d_probs, pl->fl_fwd, true, true, pl->io_forward(f[i], psi[i], op ? op[i] : nullptr),
                           nullptr, nullptr, cap);
        }
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (s != SF_OK) return s;
        if (e != cudaSuccess) return fail(SF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(SF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    SF_CK(cudaGraphLaunch(gexec, stream));
    return SF_OK;
  }

  sf_status solve_part(bool, bool, const void *, void *, void *, int *) override {
    return fail(SF_ERR_STATE, "use sf_batch_solve on a batch");
  }
  sf_status adjoint(const void *, const void *, void *) override { return fail(SF_ERR_STATE, "not available on a batch"); }
  sf_status sync() override {
    SF_CK(cudaStreamSynchronize(stream));
    bool bad = false;
    for (unsigned *flag : sticky_flags()) {
      unsigned s = 0;
      SF_CK(cudaMemcpy(&s, flag, sizeof(unsigned), cudaMemcpyDeviceToHost));
      if (s) {
        SF_CK(cudaMemset(flag, 0, sizeof(unsigned)));
        bad = true;
      }
    }
    if (bad) return fail(SF_ERR_TIMEOUT, "a scheduler wait exceeded its bound; results are invalid");
    return SF_OK;
  }
  // the batch's timeout flag and those of the fast members' executors
  std::vector<unsigned *> sticky_flags() const {
    std::vector<unsigned *> v{sticky};
    for (int i : fastm) v.push_back(plans[i]->sticky);
    return v;
  }
  sf_status query(size_t *, size_t *, size_t *, size_t *) override { return fail(SF_ERR_STATE, "query a member plan"); }
  sf_status set_face(int, int, const void *) override { return fail(SF_ERR_STATE, "not available on a batch"); }
  ExecCtl *exec_ctl() override { return ctl; }
  sf_status host_solve(const void *, void *, void *) override { return fail(SF_ERR_STATE, "not available on a batch"); }
  sf_status host_solve_many(int, const void *const *, void *const *, void *const *) override {
    return fail(SF_ERR_STATE, "not available on a batch");
  }
};

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// NVTX range around one C-ABI call (shown by nsys / ncu range filters)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

extern "C" {

const char *sf_version(void) { return "sailfish-gb300 0.1"; }

const char *sf_status_string(sf_status s) {
  switch (s) {
    case SF_OK: return "SF_OK";
    case SF_ERR_ARG: return "SF_ERR_ARG";
    case SF_ERR_UNSUPPORTED: return "SF_ERR_UNSUPPORTED";
    case SF_ERR_CUDA: return "SF_ERR_CUDA";
    case SF_ERR_OOM: return "SF_ERR_OOM";
    case SF_ERR_STATE: return "SF_ERR_STATE";
    case SF_ERR_TIMEOUT: return "SF_ERR_TIMEOUT";
    case SF_ERR_CORRUPT: return "SF_ERR_CORRUPT";
  }
  return "unknown status";
}

const char *sf_last_error(void) { return g_err.c_str(); }

sf_status sf_plan_create(sf_plan *out, const sf_plan_desc *d, void *cuda_stream) {
  NvtxRange range_("sf_plan_create");
  if (!out || !d) return fail(SF_ERR_ARG, "null argument");
  *out = nullptr;
  SF_TRY(validate(*d));
  sf_plan_s *p = nullptr;
  sf_status s;
  try {
    if (d->prec == SF_F32) {
      auto *q = new PlanImpl<float>();
      p = q;
      s = q->init(*d, (cudaStream_t)cuda_stream);
    } else {
      auto *q = new PlanImpl<double>();
      p = q;
      s = q->init(*d, (cudaStream_t)cuda_stream);
    }
  } catch (const std::exception &e) {
    delete p;
    return fail(SF_ERR_OOM, std::string("host exception: ") + e.what());
  }
  if (s != SF_OK) {
    delete p;
    return s;
  }
  *out = p;
  return SF_OK;
}

sf_status sf_plan_set_stream(sf_plan p, void *cuda_stream) {
  if (!p) return fail(SF_ERR_ARG, "null plan");
  p->stream = (cudaStream_t)cuda_stream;
  return SF_OK;
}

sf_status sf_plan_query(sf_plan p, size_t in_shape[4], size_t out_shape[4], size_t op_shape[4], size_t *ws) {
  if (!p) return fail(SF_ERR_ARG, "null plan");
  return p->query(in_shape, out_shape, op_shape, ws);
}

sf_status sf_set_source(sf_plan p, const void *dev_f) {
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (p->is_batch) return fail(SF_ERR_STATE, "not available on a batch");
  p->src = dev_f;
  return SF_OK;
}

sf_status sf_set_boundary(sf_plan p, int axis, int side, const void *dev_face) {
  if (!p) return fail(SF_ERR_ARG, "null plan");
  return p->set_face(axis, side, dev_face);
}

sf_status sf_solve(sf_plan p) {
  NvtxRange range_("sf_solve");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (p->is_batch) return fail(SF_ERR_STATE, "use sf_batch_solve on a batch");
  if (!p->src) return fail(SF_ERR_STATE, "no source set");
  SF_TRY(p->solve_part(true, false, p->src, nullptr, nullptr, nullptr));
  p->solved = true;
  return SF_OK;
}

sf_status sf_get_output(sf_plan p, void *dev_psi, void *dev_op_out) {
  NvtxRange range_("sf_get_output");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (p->is_batch) return fail(SF_ERR_STATE, "use sf_batch_solve on a batch");
  if (!p->solved) return fail(SF_ERR_STATE, "sf_get_output before sf_solve");
  if (!dev_psi) return fail(SF_ERR_ARG, "null psi");
  if (p->d.op != SF_OP_NONE && !dev_op_out) return fail(SF_ERR_ARG, "plan has an operator: op output needed");
  return p->solve_part(false, true, p->src, dev_psi, dev_op_out, nullptr);
}

sf_status sf_execute(sf_plan p, const void *dev_f, void *dev_psi, void *dev_op_out) {
  NvtxRange range_("sf_execute");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (p->is_batch) return fail(SF_ERR_STATE, "use sf_batch_solve on a batch");
  if (!dev_f || !dev_psi) return fail(SF_ERR_ARG, "null buffer");
  if (p->d.op != SF_OP_NONE && !dev_op_out) return fail(SF_ERR_ARG, "plan has an operator: op output needed");
  p->src = dev_f;
  SF_TRY(p->solve_part(true, true, dev_f, dev_psi, dev_op_out, nullptr));
  p->solved = true;
  return SF_OK;
}

sf_status sf_solve_host(sf_plan p, const void *host_f, void *host_psi, void *host_op_out) {
  NvtxRange range_("sf_solve_host");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (!host_f || !host_psi) return fail(SF_ERR_ARG, "null buffer");
  if (p->d.op != SF_OP_NONE && !host_op_out) return fail(SF_ERR_ARG, "plan has an operator: op output needed");
  return p->host_solve(host_f, host_psi, host_op_out);
}

sf_status sf_solve_host_many(sf_plan p, int n, const void *const *host_f, void *const *host_psi,
                             void *const *host_op_out) {
  NvtxRange range_("sf_solve_host_many");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (n < 0) return fail(SF_ERR_ARG, "n must be >= 0");
  if (n == 0) return SF_OK;
  if (!host_f || !host_psi) return fail(SF_ERR_ARG, "null buffer table");
  const bool need_op = p->d.op != SF_OP_NONE;
  if (need_op && !host_op_out) return fail(SF_ERR_ARG, "plan has an operator: op output table needed");
  for (int i = 0; i < n; ++i) {
    if (!host_f[i] || !host_psi[i]) return fail(SF_ERR_ARG, "null buffer in table");
    if (need_op && !host_op_out[i]) return fail(SF_ERR_ARG, "null op output in table");
  }
  return p->host_solve_many(n, host_f, host_psi, host_op_out);
}

sf_status sf_solve_adjoint(sf_plan p, const void *g_psi, const void *g_op, void *g_f) {
  NvtxRange range_("sf_solve_adjoint");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  if (!g_f) return fail(SF_ERR_ARG, "null output");
  return p->adjoint(g_psi, g_op, g_f);
}

sf_status sf_batch_create(sf_plan *batch, const sf_plan *plans, int n, void *cuda_stream) {
  NvtxRange range_("sf_batch_create");
  if (!batch || !plans || n < 1) return fail(SF_ERR_ARG, "bad batch arguments");
  *batch = nullptr;
  const int prec = plans[0] ? plans[0]->d.prec : -1;
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || plans[i]->is_batch) return fail(SF_ERR_ARG, "batch members must be plans");
    if (plans[i]->d.prec != prec) return fail(SF_ERR_UNSUPPORTED, "batch members must share the precision");
  }
  sf_plan_s *b = nullptr;
  sf_status s;
  if (prec == SF_F32) {
    auto *q = new BatchImpl<float>();
    b = q;
    s = q->init(plans, n, (cudaStream_t)cuda_stream);
  } else {
    auto *q = new BatchImpl<double>();
    b = q;
    s = q->init(plans, n, (cudaStream_t)cuda_stream);
  }
  if (s != SF_OK) {
    delete b;
    return s;
  }
  b->d = plans[0]->d;
  *batch = b;
  return SF_OK;
}

sf_status sf_batch_solve(sf_plan batch, const void *const *f, void *const *psi, void *const *op) {
  NvtxRange range_("sf_batch_solve");
  if (!batch || !batch->is_batch) return fail(SF_ERR_ARG, "not a batch");
  if (!f || !psi) return fail(SF_ERR_ARG, "null buffer table");
  if (batch->d.prec == SF_F32) return static_cast<BatchImpl<float> *>(batch)->run(f, psi, op);
  return static_cast<BatchImpl<double> *>(batch)->run(f, psi, op);
}

sf_status sf_sync(sf_plan p) {
  NvtxRange range_("sf_sync");
  if (!p) return fail(SF_ERR_ARG, "null plan");
  return p->sync();
}

int sf_plan_launches(sf_plan p) { return p ? p->launches_per_exec : 0; }

sf_status sf_selftest_timeout(int timeout_ms, void *cuda_stream) {
  if (timeout_ms < 1 || timeout_ms > 10000) return fail(SF_ERR_ARG, "timeout_ms must be in [1, 10000]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SF_TRY(set_kernel_attrs<float>());
  DevMem<float> mem;
  // a problem whose only passes are empty fills (no user data touched)
  Prob<float> q{};
  q.dim = 2;
  q.ncomp = q.nin = q.nout = 1;
  q.fill_count = 0;
  for (int a = 0; a < 3; ++a) {
    q.ax[a].kind = AK_P;
    q.ax[a].n = q.ax[a].nodes = q.ax[a].nu = q.ax[a].L = q.ax[a].ns = 1;
  }
  void *tmp;
  SF_TRY(mem.alloc(&tmp, sizeof(Prob<float>)));
  SF_CK(cudaMemcpy(tmp, &q, sizeof(Prob<float>), cudaMemcpyHostToDevice));
  const Prob<float> *dq = (const Prob<float> *)tmp;
  ExecList<float> ex;
  for (int i = 0; i < 2; ++i) {
    Pass<float> ps{};
    ps.kind = PK_FILL;
    ps.ntiles = 4;
    ps.W = ps.Wp = 1;
    ps.dep[0] = ps.dep[1] = -1;
    ex.passes.push_back(ps);
  }
  ex.passes[1].dep[0] = 0;
  ex.passes[1].depcnt[0] = ex.passes[0].ntiles + 1;  // unreachable
  SF_TRY(ex.upload(mem));
  ExecCtl *ctl;
  unsigned *sticky;
  SF_TRY(mem.alloc(&tmp, sizeof(ExecCtl)));
  ctl = (ExecCtl *)tmp;
  SF_TRY(mem.alloc(&tmp, sizeof(unsigned)));
  sticky = (unsigned *)tmp;
  SF_CK(cudaMemsetAsync(sticky, 0, sizeof(unsigned), st));
  SF_CK(cudaMemsetAsync(ex.d_done, 0, ex.passes.size() * sizeof(unsigned), st));
  SF_CK(cudaMemsetAsync(ctl, 0, sizeof(ExecCtl), st));
  IOArgs<float> io{};
  SF_CK(engine_launch_exec<float>(4, 0, st, dq, ex.d_passes, ex.d_start, (int)ex.passes.size(), ex.d_done, ctl, sticky,
                                  (unsigned long long)timeout_ms * 1000000ull, io));
  SF_CK(cudaStreamSynchronize(st));
  unsigned s = 0;
  SF_CK(cudaMemcpy(&s, sticky, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (s) return fail(SF_ERR_TIMEOUT, "scheduler wait gave up as designed");
  return SF_OK;
}

sf_status sf_eval_special(int which, int n, const double *x, double *out) {
  if (!x || !out || n < 0) return fail(SF_ERR_ARG, "null pointer or negative count");
  if (which < 0 || which > 2) return fail(SF_ERR_ARG, "unknown special function");
  for (int i = 0; i < n; ++i)
    out[i] = which == 0 ? sfg::sf_sine_integral(x[i]) : (which == 1 ? sfg::sf_int_1mj0(x[i]) : sfg::sf_expint_e1(x[i]));
  return SF_OK;
}

sf_status sf_debug_fail_alloc(int after) {
  g_alloc_budget.store(after < 0 ? -1 : (long long)after);
  return SF_OK;
}

sf_status sf_debug_corrupt_guard(sf_plan p) {
  if (!p) return fail(SF_ERR_ARG, "null plan");
  return p->corrupt_guard();
}

sf_status sf_plan_stats(sf_plan p, double out[24]) {
  if (!p || !out) return fail(SF_ERR_ARG, "null argument");
  SF_CK(cudaStreamSynchronize(p->stream));
  ExecCtl c;
  SF_CK(cudaMemcpy(&c, p->exec_ctl(), sizeof(ExecCtl), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 8; ++k) {
    out[3 * k] = (double)c.busy_ns[k];
    out[3 * k + 1] = (double)c.wait_ns[k];
    out[3 * k + 2] = (double)c.tiles[k];
  }
  return SF_OK;
}

sf_status sf_plan_timing(sf_plan p, int enable) {
  if (!p || p->is_batch) return fail(SF_ERR_ARG, "null plan or a batch");
  if (p->stream) SF_CK(cudaStreamSynchronize(p->stream));
  else SF_CK(cudaDeviceSynchronize());
  return p->timer.enable(enable != 0);
}

sf_status sf_plan_kernel_ms(sf_plan p, double ms[4], int *nslot, int *nsolve) {
  if (!p || !ms || p->is_batch) return fail(SF_ERR_ARG, "null argument or a batch");
  KernelTimer &t = p->timer;
  for (int k = 0; k < 4; ++k) ms[k] = 0.0;
  const int nsol = (int)(t.count < KernelTimer::kRing ? t.count : KernelTimer::kRing);
  const int ns = t.nmark > 1 ? t.nmark - 1 : 0;
  if (nslot) *nslot = ns;
  if (nsolve) *nsolve = nsol;
  if (!t.on || nsol == 0) return SF_OK;
  SF_CK(cudaStreamSynchronize(p->stream));
  for (int i = 0; i < nsol; ++i)
    for (int k = 0; k < ns; ++k) {
      float e = 0.f;
      SF_CK(cudaEventElapsedTime(&e, t.ev[(size_t)i * KernelTimer::kMarks + k], t.ev[(size_t)i * KernelTimer::kMarks + k + 1]));
      ms[k] += e;
    }
  for (int k = 0; k < ns; ++k) ms[k] /= nsol;
  return SF_OK;
}

sf_status sf_plan_destroy(sf_plan p) {
  if (!p) return SF_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  delete p;
  return SF_OK;
}

}  // extern "C"
