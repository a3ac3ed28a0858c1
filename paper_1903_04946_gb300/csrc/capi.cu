// capi.cu -- the C ABI of include/dso.h: context, validation, pass planning,
// operator tables, CUDA-graph replay of a composed time step.
//
// A time step of the pruned composition (Sec. II E-F) is
//   U_V(a~_1 dt) U_T(b~_1 dt) U_V(a~_2 dt) ... U_T(b~_NB dt) U_V(a~_{NB+1} dt)
// acting right to left in the paper's product, i.e. V(a~_1) first.  Each
// kinetic action needs the momentum representation (Sec. II G): a forward
// FFT over every axis, the phase, an inverse FFT over every axis.  The passes
// (kernels over whole lines of one axis, see axis_pass.cuh) run over the
// virtual axes of the grid (a grid axis longer than a pass line is two
// virtual axes, see VLayout) and are ordered so that FFTs along virtual axis
// 0 are fused with the potential step and FFTs along the last virtual axis
// with the kinetic step (Dv virtual axes):
//   Dv = 1:  [V(a~_j) F0 T(b~_j) I0] per substep, final [V(a~_{NB+1})];
//   Dv >= 2: [I0 V(a~_j) F0] [F1] .. [F_{Dv-1} T(b~_j) I_{Dv-1}] .. [I1] per
//            substep; the last potential action of a step and the first of
//            the next run in the same pass; final [I0 V(a~_{NB+1})].
// FFTs along the first factor of a split axis carry its twiddles.
// All steps after the first have the same pass list, which is captured once
// into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/dso.h"
#include "axis_pass_reg.cuh"
#include "axis_pass_tma.cuh"
#include "dso_internal.h"

using namespace dso;

namespace {

thread_local std::string g_err = "no error";

// NVTX range for the host-side extent of a library call (and the kernels it
// enqueues), for profilers: `ncu --nvtx --nvtx-include "dso_propagate/"`
// captures the kernels of propagations only.  Costs nothing without a tool.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

dso_status fail(dso_status s, const std::string& msg) {
  g_err = msg;
  return s;
}


struct Pass {
  int axis;               // virtual axis
  int SV;
  int flags;
  int u1 = -1, u2 = -1;  // potential table indices (first, second) or -1
  int tb = -1, tb2 = -1;  // kinetic table indices (first, second) or -1
};

Pass mkpass(int axis, int SV, int flags, int u1 = -1, int u2 = -1, int tb = -1, int tb2 = -1) {
  Pass p;
  p.axis = axis;
  p.SV = SV;
  p.flags = flags;
  p.u1 = u1;
  p.u2 = u2;
  p.tb = tb;
  p.tb2 = tb2;
  return p;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

struct dso_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // grid
  int D = 0;
  int64_t n[DSO_MAX_DIM] = {1, 1, 1};
  // virtual axes of the passes (VLayout), fixed when S is known
  int Dv = 0;
  int64_t nv[DSO_MAX_VAXES] = {};
  int vpart[DSO_MAX_VAXES] = {};     // 0 whole axis, 1 / 2 first / second factor of a split axis
  void* xtw[DSO_MAX_VAXES] = {};     // split twiddles [n1][n2] at the first factor's index, context precision
  double qmin[DSO_MAX_DIM] = {0, 0, 0}, qmax[DSO_MAX_DIM] = {0, 0, 0};
  double mass[DSO_MAX_DIM] = {0, 0, 0};
  bool have_grid = false, have_mass = false;
  long long P = 0;
  // model and state
  int B = 1;                 // independent jobs sharing grid, masses and scheme
  int S = 0;
  int dec0 = 0;              // surface 0 uncoupled in every job (block-diagonal potential)
  int prec = DSO_FP64;       // DSO_FP64: complex128 storage; DSO_FP32: complex64
  double* V = nullptr;       // packed [S(S+1)/2][P], always FP64
  void* psi = nullptr;       // [S][P] complex in the context's precision
  bool have_V = false, have_psi = false;
  // scheme
  int order = 2, scheme = DSO_TRIPLE_JUMP, elementary = DSO_VTV;
  Coeffs coeffs;
  bool have_coeffs = false;
  // tables for one dt
  bool tables_valid = false;
  double tables_dt = 0.0;
  void* Utab = nullptr;      // [na][S(S+1)/2][P] complex, context precision
  void* tau = nullptr;       // [nb][P] complex, context precision; separable: [nb][sum_d n_d]
  int kin_mode = DSO_KINETIC_AUTO;  // dso_set_kinetic_mode
  int boundary_merged = 1;          // dso_set_boundary_merge: one table for a~_last + a~_0
  int plane_mode = DSO_PLANE_AUTO;  // dso_set_plane_pass
  int op_mode = DSO_OPERATORS_AUTO;  // dso_set_operator_mode
  bool otf = false;                  // potential operators built per action (tables_valid: in use)
  double* eig = nullptr;             // otf: [B][eig_cache_doubles(S)][P], the coefficient-free part of U
  bool plane_on = false;            // the plan uses the plane pass (set by the autotuner)
  double* tau_a = nullptr;   // [na] potential coefficient * dt
  int n_vtab = 0, n_ttab = 0;  // numbers of potential and kinetic tables
  void* tw[14] = {};         // per log2 L (L <= 8192), context precision
  // observables
  double* Tax = nullptr;     // per-axis p^2 / (2 m_d), concatenated
  void* work = nullptr;      // [S][P] complex, context precision
  double* partials = nullptr;
  double* obs_out = nullptr;
  // norm monitor (dso_set_norm_check): tolerance (0: off), per-job norms at
  // the last dso_set_psi, device partial sums
  double norm_tol = 0.0;
  std::vector<double> norm_ref;
  double* norm_part = nullptr;
  size_t norm_part_cap = 0;  // doubles in norm_part
  // graph of one middle time step
  cudaGraphExec_t step_exec = nullptr;
  int step_exec_passes = 0;
  // tile lines and kernel variant per (axis, surfaces staged: 1 or S)
  int G[DSO_MAX_VAXES][2] = {};
  int variant[DSO_MAX_VAXES][2] = {};
  int cps[DSO_MAX_VAXES][2] = {};  // resident CTAs per SM of the persistent variants (0: as many as fit)
  int pdl = 1;               // programmatic dependent launch between passes (DSO_PDL=0: off)
  bool prev_tile = true;     // the last pass launched on the stream ran the tile kernel (variant 0)
  int wait_probe = 0;        // dso_set_wait_probe: polls of the TMA variant's diagnostic wait (0: off)
  int max_line = DSO_MAX_LINE;  // dso_set_pass_limits: longest pass line,
  int max_tile = 8192;          // and most points of the S surfaces of an axis-0 line
  bool limits_user = false;     // limits set by the caller: not tuned
  bool limits_tuned = false;    // limits chosen by timing (small 1-D grids)
  unsigned* queue = nullptr;  // tile queue of the persistent variant (2 counters)
  int* err = nullptr;         // set by kernels whose bounded waits gave up
  bool tuned = false;
  int64_t launches = 0;
  size_t esz() const { return prec == DSO_FP32 ? 8 : 16; }  // bytes per complex element
};

namespace {

void* at(void* base, size_t elems, size_t esz) { return base ? (char*)base + elems * esz : nullptr; }

int ilog2(int64_t v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

// The kinetic step as one phase per axis (each axis's phase applied between
// its own forward and inverse FFT, PASS_TAX) instead of one phase of the
// whole grid.  Needs unsplit axes (the momentum index along each line is
// that axis's own) and at least two of them.  DSO_KINETIC_AUTO takes it in
// FP32 storage mode, where it measured faster (128^3 x 3, triple jump 4:
// 0.299 against 0.322 ms per step); in FP64 the joint form is (64^3 x 3,
// Suzuki 6: 4.47 against 4.67 ms).
bool kin_axes(const dso_ctx* c) {
  const bool want = c->kin_mode == DSO_KINETIC_AXES || (c->kin_mode == DSO_KINETIC_AUTO && c->prec == DSO_FP32);
  return want && c->Dv == c->D && c->D >= 2;
}

// Length of one separable kinetic table (all axes) and the offset of axis d.
int64_t axis_table_len(const dso_ctx* c) {
  int64_t n = 0;
  for (int d = 0; d < c->D; ++d) n += c->n[d];
  return n;
}

int64_t axis_table_off(const dso_ctx* c, int d) {
  int64_t n = 0;
  for (int e = 0; e < d; ++e) n += c->n[e];
  return n;
}

// The plane pass (the kinetic passes of axes 1 and 2 in one launch: [F1 T1
// I1 | F2 T2 I2] per axis, [F1 | F2 T I2 | I1] joint) applies to a 3-D grid of
// whole axes whose two last axes are register-resident line lengths;
// plane_on is the tuned choice.
bool plane_supported(const dso_ctx* c) {
  return c->D == 3 && c->Dv == 3 && c->plane_mode != DSO_PLANE_OFF &&
         axis_pass_plane_supported((int)c->nv[1], (int)c->nv[2], c->prec == DSO_FP32);
}

bool plane_active(const dso_ctx* c) { return c->plane_on && plane_supported(c); }

// Step boundaries.  A symmetric composition's last a~ action of one step and
// first of the next act back to back on the same operator (the potential in
// VTV, the kinetic step in TVT), so they are one action with coefficient
// a~_last + a~_0 (Sec. II F merges adjacent actions of one operator the same
// way).  With boundary_merged that action has a table of its own: the index
// of a~_last + a~_0 among the unique a~ values (equal to a relative 1e-12, as
// the unique values are found), or one past them when it is new.  -1: the two
// actions are applied one after the other in one pass.
int merged_a_index(const dso_ctx* c) {
  if (!c->boundary_merged || c->coeffs.a.empty()) return -1;
  const double m = c->coeffs.a.front() + c->coeffs.a.back();
  const std::vector<double>& u = c->coeffs.a_unq;
  for (size_t j = 0; j < u.size(); ++j)
    if (std::fabs(u[j] - m) <= 1e-12 * std::fabs(m)) return (int)j;
  return (int)u.size();
}

// The a~ values with tables: the unique ones, plus the merged boundary value
// when it is new.
std::vector<double> a_table_values(const dso_ctx* c) {
  std::vector<double> v = c->coeffs.a_unq;
  const int mi = merged_a_index(c);
  if (mi == (int)v.size()) v.push_back(c->coeffs.a.front() + c->coeffs.a.back());
  return v;
}

void drop_graph(dso_ctx* c) {
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  c->step_exec = nullptr;
  c->step_exec_passes = 0;
}

void drop_tables(dso_ctx* c) {
  drop_graph(c);
  dfree(c->Utab);
  dfree(c->eig);
  dfree(c->tau);
  dfree(c->tau_a);
  c->tables_valid = false;
  c->otf = false;
}

// Potential table slots per job: one per unique coefficient, or (operators
// built per action) two, the pass's first and second table.
int vslots(const dso_ctx* c) { return c->otf ? 2 : c->n_vtab; }

void drop_model(dso_ctx* c) {
  drop_tables(c);
  c->tuned = false;
  dfree(c->V);
  dfree(c->psi);
  dfree(c->Tax);
  dfree(c->work);
  dfree(c->partials);
  dfree(c->obs_out);
  dfree(c->norm_part);
  c->norm_part_cap = 0;
  for (auto& x : c->xtw) dfree(x);
  c->norm_ref.clear();
  c->have_V = c->have_psi = false;
}

// Virtual axes of the passes for the grid and S surfaces (VLayout): a grid
// axis longer than a pass line (max_line), or an axis 0 whose S surfaces do
// not fit the potential pass's tile (S n > max_tile), is split into
// n1 = 2^floor(log2(n) / 2) (halved further on axis 0 until S n1 <= max_tile)
// and n2 = n / n1.  With the default limits (4096, 8192) every axis up to 2^22
// points splits into factors <= 2048 and S n1 <= 8192 for every S <= 4; with
// tighter limits a grid may not fit, and the plan fails (false).
bool plan_virtual(dso_ctx* c) {
  c->Dv = 0;
  for (int d = 0; d < c->D; ++d) {
    const int64_t n = c->n[d];
    if (n > c->max_line || (d == 0 && (long long)c->S * n > c->max_tile)) {
      int64_t n1 = 1LL << (ilog2(n) / 2);
      while (d == 0 && (long long)c->S * n1 > c->max_tile && n1 > 8) n1 /= 2;
      const int64_t n2 = n / n1;
      if (n1 < 8 || n2 < 8 || n1 > c->max_line || n2 > c->max_line ||
          (d == 0 && (long long)c->S * n1 > c->max_tile))
        return false;
      c->nv[c->Dv] = n1;
      c->vpart[c->Dv++] = 1;
      c->nv[c->Dv] = n2;
      c->vpart[c->Dv++] = 2;
    } else {
      c->nv[c->Dv] = n;
      c->vpart[c->Dv++] = 0;
    }
  }
  return true;
}

VLayout vlayout(const dso_ctx* c) {
  VLayout v{};
  v.Dv = c->Dv;
  for (int a = 0; a < DSO_MAX_VAXES; ++a) {
    v.nv[a] = a < c->Dv ? c->nv[a] : 1;
    v.part[a] = a < c->Dv ? c->vpart[a] : 0;
  }
  v.D = c->D;
  for (int d = 0; d < 3; ++d) v.n[d] = c->n[d];
  return v;
}

// Line length of the passes along virtual axis d.
int kind_L(const dso_ctx* c, int d, int /*which*/) { return (int)c->nv[d]; }

// Tile lines per surface for a pass over lines of length L staging SV
// surfaces: the largest power of two giving at most about 128 threads
// (8 values each) per CTA, so that many CTAs share each SM and the last wave
// is short.  A power of two always divides the line count and either divides
// the axis stride or is a multiple of it, which the tile geometry relies on.
int choose_G(const dso_ctx* c, int L, int SV) {
  const long long lines = c->P / L;
  const long long target = (128LL * 8) / ((long long)SV * L);
  const long long gmax = axis_pass_max_tile_lines(L, SV);
  long long G = 1;
  while (G * 2 <= target && G * 2 <= gmax && G * 2 <= lines) G *= 2;
  return (int)G;
}

// (Re)plan the virtual axes of a context whose S is known, and reset the
// per-kind tile line counts and kernel variants (the tables, graph and
// tuning that depend on the layout are dropped).
dso_status replan(dso_ctx* c) {
  if (!plan_virtual(c)) return fail(DSO_EINVAL, "the grid does not fit the pass limits (a split factor exceeds them)");
  for (int d = 0; d < c->Dv; ++d) {
    // every pass line fits one tile: S surfaces of a virtual axis-0 line,
    // one surface of any other
    if (!axis_pass_supported((int)c->nv[d], d == 0 ? c->S : 1))
      return fail(DSO_EINVAL, "internal: a pass line does not fit a tile");
    c->G[d][0] = choose_G(c, (int)c->nv[d], 1);
    c->G[d][1] = choose_G(c, (int)c->nv[d], c->S);
    c->variant[d][0] = c->variant[d][1] = 0;
    c->cps[d][0] = c->cps[d][1] = 0;
  }
  for (auto& x : c->xtw) dfree(x);
  drop_tables(c);
  c->tuned = false;
  return DSO_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &f, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 5-D FP64 view (re/im, inner i, line position n, outer o, block) of a
// [blocks][P] complex array for lines along an axis of length L and stride
// `stride`; box {2, Wi, L, Go, bbox}.
bool encode_view(CUtensorMap* m, const void* base, long long P, int L, long long stride, long long blocks, int Wi,
                 int Go, int bbox) {
  auto fn = encode_fn();
  if (!fn) return false;
  const long long outer = P / ((long long)L * stride);
  cuuint64_t dims[5] = {2, (cuuint64_t)stride, (cuuint64_t)L, (cuuint64_t)outer, (cuuint64_t)blocks};
  cuuint64_t strides[4] = {16, (cuuint64_t)(16 * stride), (cuuint64_t)(16 * stride * L), (cuuint64_t)(16 * P)};
  cuuint32_t box[5] = {2, (cuuint32_t)Wi, (cuuint32_t)L, (cuuint32_t)Go, (cuuint32_t)bbox};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The kernel arguments of pass p (and the number of its tiles), with the
// tile line count the context holds for the pass's kind.
cudaError_t build_pass_args(dso_ctx* c, const Pass& p, PassArgs& a, long long& ntiles) {
  const int L = (int)c->nv[p.axis];
  a = PassArgs{};  // every field defined; the kernels read all of them
  const size_t es = c->esz();
  a.psi = c->psi;
  const int NP = c->S * (c->S + 1) / 2;
  // operators built per action: the pass reads slot 0 (first table) and
  // slot 1 (second), which run_pass fills before launching it
  const int s1 = c->otf ? (p.u1 >= 0 ? 0 : -1) : p.u1, s2 = c->otf ? (p.u2 >= 0 ? 1 : -1) : p.u2;
  a.U1 = s1 >= 0 ? at(c->Utab, (size_t)s1 * NP * c->P, es) : nullptr;
  a.U2 = s2 >= 0 ? at(c->Utab, (size_t)s2 * NP * c->P, es) : nullptr;
  a.fp32 = c->prec == DSO_FP32 ? 1 : 0;
  if (p.flags & PASS_TAX) {  // this axis's phase: [nb][sum_d n_d] tables, 1/L folded in
    const size_t len = (size_t)axis_table_len(c), off = (size_t)axis_table_off(c, p.axis);
    a.tau = p.tb >= 0 ? at(c->tau, (size_t)p.tb * len + off, es) : nullptr;
    a.tau2 = p.tb2 >= 0 ? at(c->tau, (size_t)p.tb2 * len + off, es) : nullptr;
    a.tau2_scale = (double)L;
  } else {
    a.tau = p.tb >= 0 ? at(c->tau, (size_t)p.tb * c->P, es) : nullptr;
    a.tau2 = p.tb2 >= 0 ? at(c->tau, (size_t)p.tb2 * c->P, es) : nullptr;
    a.tau2_scale = (double)c->P;
  }
  a.tw = c->tw[ilog2(L)];
  if (!a.tw) return cudaErrorInvalidValue;  // no twiddle table for this line length
  a.P = c->P;
  long long stride = 1;
  for (int d = p.axis + 1; d < c->Dv; ++d) stride *= c->nv[d];
  a.stride = stride;
  a.lines = c->P / L;
  a.S = c->S;
  const int which = p.SV == 1 ? 0 : 1;
  a.G = c->G[p.axis][which];
  a.flags = p.flags;
  if (c->vpart[p.axis] == 1 && (p.flags & (PASS_INV_FIRST | PASS_FWD))) {
    // FFTs along the first factor of a split axis carry the four-step twiddles
    if (p.flags & PASS_T) return cudaErrorInvalidConfiguration;  // never planned
    a.flags |= PASS_XTW;
    a.xtw = c->xtw[p.axis];
    a.xtw_n2_log2 = ilog2(c->nv[p.axis + 1]);
    a.xtw_s2_log2 = ilog2(stride / c->nv[p.axis + 1]);
    if (!a.xtw) return cudaErrorInvalidValue;
  }
  if (a.G < 1 || (a.G & (a.G - 1)) || a.lines % a.G) return cudaErrorInvalidConfiguration;
  a.stride_log2 = ilog2(stride);
  a.G_log2 = ilog2(a.G);
  a.ua = s1 >= 0 ? s1 : 0;
  a.ub = p.tb >= 0 ? p.tb : 0;
  a.err = c->err;
  a.nbatch = c->B;
  a.u_batch_stride = (long long)vslots(c) * NP * c->P;
  a.U_base = c->Utab;
  a.tau_base = c->tau;
  a.psi_elems = (long long)c->B * c->S * c->P;
  a.u_elems = (long long)c->B * vslots(c) * NP * c->P;
  a.tau_elems = (long long)c->n_ttab * (kin_axes(c) ? axis_table_len(c) : c->P);
  a.dec0 = c->dec0;
  a.ctas_per_sm = c->cps[p.axis][which];
  a.pdl = c->pdl;
  a.wait_probe = c->wait_probe;
  ntiles = (p.SV == c->S) ? (long long)c->B * (a.lines / a.G) : (long long)c->B * c->S * (a.lines / a.G);
  if (p.flags & PASS_PLANE) {  // one plane of axes 1 and 2 of one surface per cluster
    if (c->Dv != 3 || p.axis != 1 || p.SV != 1) return cudaErrorInvalidConfiguration;
    a.tw2 = c->tw[ilog2(c->nv[2])];
    if (!a.tw2) return cudaErrorInvalidValue;
    ntiles = (long long)c->B * c->S * c->nv[0];
  }
  return cudaSuccess;
}

// Operators built per action: fill slot 0 (and 1) of every job with the
// pass's potential table(s) from the stored coefficient-free part.  The
// passes stage their tables before waiting for the previous kernel, so the
// pass that follows is launched without programmatic dependent launch.
cudaError_t build_operator_slots(dso_ctx* c, const Pass& p) {
  const int NP = c->S * (c->S + 1) / 2;
  const size_t nc = (size_t)eig_cache_doubles(c->S);
  const int coef[2] = {p.u1, p.u2};
  for (int k = 0; k < 2; ++k) {
    if (coef[k] < 0) continue;
    if (coef[k] >= c->n_vtab) return cudaErrorInvalidValue;
    for (int b = 0; b < c->B; ++b) {
      const cudaError_t e =
          launch_unitary_from_cache(at(c->Utab, ((size_t)b * 2 + k) * NP * c->P, c->esz()), c->prec == DSO_FP32,
                                    c->eig + (size_t)b * nc * c->P, c->tau_a + coef[k], c->S, c->P, c->stream);
      if (e != cudaSuccess) return e;
      c->launches += 1;
    }
  }
  c->prev_tile = true;  // no programmatic dependent launch for the next pass
  return cudaSuccess;
}

cudaError_t run_pass(dso_ctx* c, const Pass& p) {
  const int L = (int)c->nv[p.axis];
  PassArgs a;
  long long ntiles = 0;
  {
    const cudaError_t e = build_pass_args(c, p, a, ntiles);
    if (e != cudaSuccess) return e;
  }
  if (c->otf && p.u1 >= 0) {
    const cudaError_t e = build_operator_slots(c, p);
    if (e != cudaSuccess) return e;
  }
  if (p.flags & PASS_PLANE) {  // one kernel, no variants; PDL as between the non-tile variants
    if (c->prev_tile) a.pdl = 0;
    c->prev_tile = false;
    c->launches += 1;
    return launch_axis_pass_plane(L, (int)c->nv[2], a, ntiles, c->stream);
  }
  const long long stride = a.stride;
  const int which = p.SV == 1 ? 0 : 1;
  const int variant = c->variant[p.axis][which];
  TmaMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  if (variant == 3 && p.u1 >= 0 && p.tb >= 0) return cudaErrorInvalidConfiguration;  // 1-D passes
  if ((variant == 2 || variant == 3) && (p.flags & PASS_TAX)) return cudaErrorInvalidConfiguration;
  if (variant == 2 || variant == 3) {
    const int Wi = (int)(stride < a.G ? stride : a.G);
    const int Go = a.G / Wi;
    const int NP = c->S * (c->S + 1) / 2;
    bool ok = encode_view(&maps.psi, c->psi, c->P, L, stride, (long long)c->B * c->S, Wi, Go, p.SV);
    if (ok && p.u1 >= 0)
      ok = encode_view(&maps.tab, c->Utab, c->P, L, stride, (long long)c->B * NP * (long long)vslots(c), Wi, Go,
                       NP);
    if (ok && p.tb >= 0) {
      CUtensorMap* m = (p.u1 >= 0) ? &maps.tab2 : &maps.tab;
      ok = encode_view(m, c->tau, c->P, L, stride, (long long)c->n_ttab, Wi, Go, 1);
    }
    // every box the kernel will address must lie inside its tensor
    const long long outer = c->P / ((long long)L * stride);
    const long long t_per_set = a.lines / a.G;
    const long long i_last = ((t_per_set - 1) * a.G) % stride, o_last = ((t_per_set - 1) * a.G) / stride;
    if (i_last + Wi > stride || o_last + Go > outer) ok = false;
    if (p.u1 >= 0 && ((long long)(c->B - 1) * vslots(c) * NP + (long long)a.ua * NP + NP >
                      (long long)c->B * vslots(c) * NP))
      ok = false;
    if (p.tb >= 0 && p.tb >= c->n_ttab) ok = false;
    if (!ok) return cudaErrorInvalidConfiguration;
  }
  c->launches += 1;
  // Programmatic dependent launch only between two passes of the other
  // variants: the tile kernel's many small CTAs measured slower with it on
  // either side (64^3 x 3 FP64: all tile passes 4.46 -> 5.93 ms per step; a
  // tile kinetic pass between register-resident ones 4.45 -> 4.9 ms), while a
  // step of TMA and register-resident passes gains from it (4.54 -> 4.31 ms).
  if (variant == 0 || c->prev_tile) a.pdl = 0;
  c->prev_tile = variant == 0;
  return launch_axis_pass(L, p.SV, variant, a, ntiles, c->queue, &maps, c->stream);
}

// Pass lists.  VTV (Eq. (so_VTV)): the potential acts first and last, with
// tables indexed by I^a and kinetic tables by I^b.  TVT (Eq. (so_TVT)): the
// kinetic step acts first and last, with kinetic tables indexed by I^a and
// potential tables by I^b.  The list of a middle step is the same for every
// step after the first, so it is captured once in a CUDA graph.
//
// VTV, D >= 2:  [I0 V F0] [F1..] [F_{D-1} T I_{D-1}] [..I1] per substep,
//   final [I0 V]; at step boundaries the last V of a step and the first of
//   the next share one pass.
// VTV, D = 1:   [V F0 T I0] per substep, final [V].
// TVT, D >= 2:  first step starts with a standalone [F0]; every potential
//   action is [I0 V F0]; the last kinetic action of a step and the first of
//   the next share one kinetic pass; final kinetic action then [I0].
// TVT, D = 1:   [F0 T I0], then [V F0 T I0] per substep; the final pass is
//   [V F0 T I0] with the step's last coefficients.
// With the plane pass (plane_active, D = 3) [F1] [F2 T I2] [I1] is one pass,
// [F1 | F2 T I2 | I1].
void t_action(const dso_ctx* c, std::vector<Pass>& out, bool standalone_f0, int tb, int tb2) {
  const int D = c->Dv;
  if (standalone_f0) out.push_back(mkpass(0, 1, PASS_FWD));
  if (plane_active(c)) {  // [F1 | F2 T I2 | I1]: the plane pass
    out.push_back(mkpass(1, 1, PASS_FWD | PASS_T | PASS_PLANE, -1, -1, tb, tb2));
    return;
  }
  for (int d = 1; d <= D - 2; ++d) out.push_back(mkpass(d, 1, PASS_FWD));
  out.push_back(mkpass(D - 1, 1, PASS_FWD | PASS_T, -1, -1, tb, tb2));
  for (int d = D - 2; d >= 1; --d) out.push_back(mkpass(d, 1, PASS_INV_FIRST));
}

// Separable kinetic step (kin_axes), D >= 2: every kinetic action is one
// pass [F_d T_d I_d] per axis, each applying that axis's phase between its own
// FFTs; the potential action joins the axis-0 pass of the next kinetic action.
// VTV:  [V F0 T0 I0] [F1 T1 I1] .. [F_{D-1} T_{D-1} I_{D-1}] per substep,
//   final [V]; at step boundaries the last V of a step and the first of the
//   next share one pass.
// TVT:  [F0 T0 I0] .. in the first substep of the first step, then [V F0 T0
//   I0] ..; at step boundaries both kinetic coefficients' phases act in one
//   pass per axis; the final kinetic action is [V F0 T0 I0] .. with the
//   step's last coefficients.
// With the plane pass (plane_active, D = 3) the passes of axes 1 and 2 are
// one: [V F0 T0 I0] [F1 T1 I1 | F2 T2 I2].
void t_action_axes(const dso_ctx* c, std::vector<Pass>& out, int u1, int u2, int tb, int tb2) {
  const int f = PASS_FWD | PASS_T | PASS_TAX;
  out.push_back(mkpass(0, u1 >= 0 ? c->S : 1, f, u1, u2, tb, tb2));
  if (plane_active(c)) {  // [F1 T1 I1 | F2 T2 I2]: the plane pass
    out.push_back(mkpass(1, 1, f | PASS_PLANE, -1, -1, tb, tb2));
    return;
  }
  for (int d = 1; d < c->Dv; ++d) out.push_back(mkpass(d, 1, f, -1, -1, tb, tb2));
}

std::vector<Pass> step_passes_axes(const dso_ctx* c, bool first) {
  std::vector<Pass> out;
  const std::vector<int>& ia = c->coeffs.ia;
  const std::vector<int>& ib = c->coeffs.ib;
  const int NB = (int)c->coeffs.b.size();
  const int last = (int)c->coeffs.a.size() - 1;
  for (int j = 0; j < NB; ++j) {
    if (c->elementary == DSO_VTV) {
      const bool merge = j == 0 && !first;
      const int mi = merged_a_index(c);
      if (merge && mi >= 0)
        t_action_axes(c, out, mi, -1, ib[j], -1);
      else
        t_action_axes(c, out, merge ? ia[last] : ia[j], merge ? ia[0] : -1, ib[j], -1);
    } else {
      const bool merge = j == 0 && !first;
      const int uv = (j == 0) ? (first ? -1 : ib[NB - 1]) : ib[j - 1];
      const int mi = merged_a_index(c);
      if (merge && mi >= 0)
        t_action_axes(c, out, uv, -1, mi, -1);
      else
        t_action_axes(c, out, uv, -1, merge ? ia[last] : ia[j], merge ? ia[0] : -1);
    }
  }
  return out;
}

std::vector<Pass> final_passes_axes(const dso_ctx* c) {
  std::vector<Pass> out;
  const int last = (int)c->coeffs.a.size() - 1;
  const int NB = (int)c->coeffs.b.size();
  if (c->elementary == DSO_VTV)
    out.push_back(mkpass(0, c->S, 0, c->coeffs.ia[last]));
  else
    t_action_axes(c, out, c->coeffs.ib[NB - 1], -1, c->coeffs.ia[last], -1);
  return out;
}

std::vector<Pass> step_passes(const dso_ctx* c, bool first) {
  if (kin_axes(c)) return step_passes_axes(c, first);
  std::vector<Pass> out;
  const std::vector<int>& ia = c->coeffs.ia;
  const std::vector<int>& ib = c->coeffs.ib;
  const int NB = (int)c->coeffs.b.size();
  const int last = (int)c->coeffs.a.size() - 1;  // = NB
  const int D = c->Dv;
  if (c->elementary == DSO_VTV) {
    for (int j = 0; j < NB; ++j) {
      int u1 = ia[j], u2 = -1;
      if (j == 0 && !first) {
        const int mi = merged_a_index(c);
        u1 = mi >= 0 ? mi : ia[last];
        u2 = mi >= 0 ? -1 : ia[0];
      }
      if (D == 1) {
        out.push_back(mkpass(0, c->S, PASS_FWD | PASS_T, u1, u2, ib[j]));
        continue;
      }
      const int inv_first = (j == 0 && first) ? 0 : PASS_INV_FIRST;
      out.push_back(mkpass(0, c->S, inv_first | PASS_FWD, u1, u2));
      t_action(c, out, false, ib[j], -1);
    }
    return out;
  }
  // TVT: kinetic coefficients a~ (tables by I^a), potential b~ (tables by I^b)
  for (int j = 0; j < NB; ++j) {
    const int mi = merged_a_index(c);
    const bool merge = j == 0 && !first;
    const int tb = merge ? (mi >= 0 ? mi : ia[last]) : ia[j];
    const int tb2 = (merge && mi < 0) ? ia[0] : -1;
    const int uv = (j == 0) ? (first ? -1 : ib[NB - 1]) : ib[j - 1];
    if (D == 1) {
      out.push_back(mkpass(0, c->S, PASS_FWD | PASS_T, uv, -1, tb, tb2));
      continue;
    }
    if (uv >= 0) out.push_back(mkpass(0, c->S, PASS_INV_FIRST | PASS_FWD, uv));
    t_action(c, out, uv < 0, tb, tb2);
  }
  return out;
}

std::vector<Pass> final_passes(const dso_ctx* c) {
  if (kin_axes(c)) return final_passes_axes(c);
  std::vector<Pass> out;
  const int last = (int)c->coeffs.a.size() - 1;
  const int NB = (int)c->coeffs.b.size();
  if (c->elementary == DSO_VTV) {
    out.push_back(mkpass(0, c->S, c->Dv == 1 ? 0 : PASS_INV_FIRST, c->coeffs.ia[last]));
    return out;
  }
  const int uv = c->coeffs.ib[NB - 1];
  if (c->Dv == 1) {
    out.push_back(mkpass(0, c->S, PASS_FWD | PASS_T, uv, -1, c->coeffs.ia[last]));
    return out;
  }
  out.push_back(mkpass(0, c->S, PASS_INV_FIRST | PASS_FWD, uv));
  t_action(c, out, false, c->coeffs.ia[last], -1);
  out.push_back(mkpass(0, 1, PASS_INV_FIRST));
  return out;
}

#define CK(expr)                                                                                  \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess)                                                                        \
      return fail(_e == cudaErrorMemoryAllocation ? DSO_ENOMEM : DSO_ECUDA,                       \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                            \
  } while (0)

dso_status ensure_twiddles(dso_ctx* c) {
  // the FFT twiddles of every line length a pass uses (the virtual axis
  // lengths), and the four-step twiddles of every split axis
  std::vector<int> lens;
  for (int d = 0; d < c->Dv; ++d) lens.push_back((int)c->nv[d]);
  for (int d = 0; d + 1 < c->Dv; ++d) {
    if (c->vpart[d] != 1 || c->xtw[d]) continue;
    const int64_t n = c->nv[d] * c->nv[d + 1];
    CK(cudaMalloc(&c->xtw[d], (size_t)n * c->esz()));
    CK(launch_split_twiddles(c->xtw[d], c->prec == DSO_FP32, c->nv[d], c->nv[d + 1], c->stream));
    c->launches += 1;
  }
  for (int L : lens) {
    const int l = ilog2(L);
    if (c->tw[l]) continue;
    std::vector<double2> h = host_twiddles(L, c->prec == DSO_FP32);
    if (c->prec == DSO_FP32) {
      std::vector<float2> hf(h.size());
      for (size_t i = 0; i < h.size(); ++i) hf[i] = make_float2((float)h[i].x, (float)h[i].y);
      CK(cudaMalloc(&c->tw[l], hf.size() * sizeof(float2)));
      CK(cudaMemcpy(c->tw[l], hf.data(), hf.size() * sizeof(float2), cudaMemcpyHostToDevice));
    } else {
      CK(cudaMalloc(&c->tw[l], h.size() * sizeof(double2)));
      CK(cudaMemcpy(c->tw[l], h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
  }
  return DSO_OK;
}

// allow_otf = false (batch slots, whose work-list kernel reads tables only)
// keeps the precomputed tables whatever the operator mode.
dso_status ensure_tables(dso_ctx* c, double dt, bool allow_otf = true) {
  if (!allow_otf && c->op_mode == DSO_OPERATORS_ON_THE_FLY)
    return fail(DSO_EINVAL, "operators built per action (DSO_OPERATORS_ON_THE_FLY) are not available in a batch slot");
  if (c->tables_valid && c->tables_dt == dt && (allow_otf || !c->otf)) return DSO_OK;
  NvtxRange nvtx("dso_tables");
  CK(cudaGetLastError());  // surface any error left pending by an earlier call
  drop_tables(c);
  dso_status st = ensure_twiddles(c);
  if (st != DSO_OK) return st;
  // VTV: the potential takes the a~ coefficients and the kinetic step the b~;
  // TVT swaps them.
  const std::vector<double> avals = a_table_values(c);
  const std::vector<double>& vco = (c->elementary == DSO_VTV) ? avals : c->coeffs.b_unq;
  const std::vector<double>& tco = (c->elementary == DSO_VTV) ? c->coeffs.b_unq : avals;
  const int na = (int)vco.size(), nb = (int)tco.size();
  const int NP = c->S * (c->S + 1) / 2;
  // Sec. II F's memory/time trade-off: one potential table per unique
  // coefficient, or (operators built per action) the coefficient-free part
  // of U per point and two table slots filled before each potential pass.
  // DSO_OPERATORS_AUTO builds the tables when they take at most half the
  // free device memory.
  const size_t table_bytes = (size_t)c->B * na * NP * c->P * c->esz();
  bool otf = c->op_mode == DSO_OPERATORS_ON_THE_FLY;
  if (c->op_mode == DSO_OPERATORS_AUTO && allow_otf) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    otf = table_bytes > free_b / 2;
  }
  c->otf = otf;
  CK(cudaMalloc(&c->Utab, otf ? (size_t)c->B * 2 * NP * c->P * c->esz() : table_bytes));
  const bool sep = kin_axes(c);
  CK(cudaMalloc(&c->tau, (size_t)nb * (sep ? axis_table_len(c) : c->P) * c->esz()));
  CK(cudaMalloc(&c->tau_a, (size_t)na * sizeof(double)));
  c->n_vtab = na;
  c->n_ttab = nb;
  std::vector<double> ta(na);
  for (int u = 0; u < na; ++u) ta[u] = vco[u] * dt;
  CK(cudaMemcpyAsync(c->tau_a, ta.data(), na * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaGetLastError());
  if (otf) {
    const size_t nc = (size_t)eig_cache_doubles(c->S);
    CK(cudaMalloc(&c->eig, (size_t)c->B * nc * c->P * sizeof(double)));
    for (int b = 0; b < c->B; ++b) {
      CK(launch_eig_cache(c->eig + (size_t)b * nc * c->P, c->V + (size_t)b * NP * c->P, c->S, c->P, c->stream));
      c->launches += 1;
    }
  } else {
    for (int b = 0; b < c->B; ++b) {
      CK(launch_potential_tables(at(c->Utab, (size_t)b * na * NP * c->P, c->esz()), c->prec == DSO_FP32,
                                 c->V + (size_t)b * NP * c->P, c->tau_a, na, c->S, c->P, c->stream));
      c->launches += 1;
    }
  }
  std::vector<double> coef = host_kinetic_coefficients(c->D, c->qmin, c->qmax, c->mass, tco, dt);
  double* dcoef = nullptr;
  CK(cudaMalloc(&dcoef, coef.size() * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(dcoef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = sep ? launch_axis_kinetic_tables(c->tau, c->prec == DSO_FP32, dcoef, nb, c->D, c->n, c->stream)
            : launch_kinetic_tables(c->tau, c->prec == DSO_FP32, dcoef, nb, vlayout(c), c->P, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dcoef);
  CK(e);
  c->launches += 1;
  c->tables_valid = true;
  c->tables_dt = dt;
  return DSO_OK;
}

// Tile-size autotuner.  For every kind of pass the propagation uses, time
// each admissible tile line count G (a power of two whose CTA is a whole
// number of warps, when one exists) with CUDA events on a copy of psi and the
// real operator tables, and keep the fastest.  The FFT work per amplitude
// does not depend on G; G trades load balance across the SMs (many small
// CTAs) against per-CTA overhead.  Skipped when DSO_AUTOTUNE=0.
// Tuning results are shared by every context of the process with the same
// grid, surface count, batch, precision and elementary method, so that a
// stream of jobs of one shape (a serving loop) tunes once.
// The key holds everything that fixes the pass kinds and their lines: the
// grid, S (which with the pass limits fixes the virtual axes), the batch,
// precision, elementary method, device, the form of the kinetic step, the
// plane-pass mode and whether the potential operators are built per action.
using TuneKey = std::tuple<int, int64_t, int64_t, int64_t, int, int, int, int, int, int, int, int, int, int>;
struct TuneVal {
  int G[DSO_MAX_VAXES][2];
  int variant[DSO_MAX_VAXES][2];
  int cps[DSO_MAX_VAXES][2];
  int plane;  // plane pass chosen
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

TuneKey tune_key(const dso_ctx* c) {
  return TuneKey(c->D, c->n[0], c->n[1], c->n[2], c->S, c->B, c->prec, c->elementary, c->device, c->max_line,
                 c->max_tile, kin_axes(c) ? 1 : 0, c->plane_mode, c->otf ? 1 : 0);
}

dso_status autotune_tiles(dso_ctx* c) {
  if (c->tuned) return DSO_OK;
  NvtxRange nvtx("dso_autotune");
  c->plane_on = c->plane_mode == DSO_PLANE_ON;  // DSO_PLANE_AUTO: chosen below by timing
  // a fixed configuration (DSO_PLAN, as written by dso_tuned_plan)
  if (const char* plan = getenv("DSO_PLAN")) {
    const char* q = plan;
    int d, w, v, g, cp, used;
    while (sscanf(q, "%d,%d,%d,%d,%d;%n", &d, &w, &v, &g, &cp, &used) == 5) {
      q += used;
      if (d < 0 || d >= c->Dv || w < 0 || w > 1 || v < 0 || v > 4 || g < 1 || (g & (g - 1))) continue;
      if (c->vpart[d] == 1 && v != 0) continue;  // split-axis twiddles: tile kernel only
      const long long L = kind_L(c, d, w), lines = c->P / L;
      const int SV = w ? c->S : 1;
      if (lines % g) continue;
      if (v == 4 ? g != axis_pass_reg_lines((int)L, SV) : g > axis_pass_max_tile_lines((int)L, SV)) continue;
      if (v == 4) {
        long long stride = 1;
        for (int e = d + 1; e < c->Dv; ++e) stride *= c->nv[e];
        if (!axis_pass_reg_supported((int)L, SV, c->prec == DSO_FP32, stride, c->dec0 != 0)) continue;
      }
      if (c->prec == DSO_FP32 && v != 0 && v != 4) continue;
      if ((v == 1 && !axis_pass_pq_supported((int)L, SV, g)) || (v == 2 && !axis_pass_tma_supported((int)L, SV, g)) ||
          (v == 3 && (!axis_pass_tmap_supported((int)L, SV, g) || c->Dv == 1)))
        continue;
      c->G[d][w] = g;
      c->variant[d][w] = v;
      c->cps[d][w] = cp < 0 ? 0 : cp;
    }
    // a trailing "plane;" selects the plane pass (unless DSO_PLANE_OFF)
    if (std::strncmp(q, "plane;", 6) == 0) c->plane_on = true;
    c->tuned = true;
    return DSO_OK;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(c));
    if (it != g_tune_cache.end() && !getenv("DSO_VARIANT")) {
      std::memcpy(c->G, it->second.G, sizeof(c->G));
      std::memcpy(c->variant, it->second.variant, sizeof(c->variant));
      std::memcpy(c->cps, it->second.cps, sizeof(c->cps));
      c->plane_on = it->second.plane != 0;
      c->tuned = true;
      return DSO_OK;
    }
  }
  const char* env = getenv("DSO_AUTOTUNE");
  const char* fv0 = getenv("DSO_VARIANT");
  if (env && env[0] == '0' && !(fv0 && fv0[0])) {
    c->tuned = true;
    return DSO_OK;
  }
  if (!c->work) CK(cudaMalloc(&c->work, (size_t)c->B * c->S * c->P * c->esz()));
  CK(cudaMemcpyAsync(c->work, c->psi, (size_t)c->B * c->S * c->P * c->esz(), cudaMemcpyDeviceToDevice,
                     c->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  void* keep = c->psi;
  c->psi = c->work;
  const int64_t launches = c->launches;
  // every kind of pass (axis, surfaces staged) the propagation uses, with a
  // representative pass of that kind: from a middle step where the kind
  // occurs there (the passes every later step repeats, e.g. [I0 V F0] rather
  // than the first step's [V F0]), else from the first step or the final
  // passes
  std::vector<Pass> plan = step_passes(c, false);
  for (const Pass& q : step_passes(c, true)) plan.push_back(q);
  for (const Pass& q : final_passes(c)) plan.push_back(q);
  std::vector<Pass> reps;
  bool both[DSO_MAX_VAXES][2] = {};  // some pass of the kind applies a potential and a kinetic phase (1-D)
  for (const Pass& q : plan)
    if (q.u1 >= 0 && q.tb >= 0) both[q.axis][q.SV == 1 ? 0 : 1] = true;
  for (const Pass& q : plan) {
    if (q.flags & PASS_PLANE) continue;  // one kernel: nothing to tune
    bool seen = false;
    for (const Pass& r : reps)
      if (r.axis == q.axis && (r.SV == 1) == (q.SV == 1)) seen = true;
    if (!seen) reps.push_back(q);
  }
  TuneVal alt[2] = {};  // whole-step candidates: tile kernel everywhere; the other variants where they apply
  // fastest time alone, and its tile lines and CTAs per SM, of every variant of every kind
  float vbest[DSO_MAX_VAXES][2][5];
  int vG[DSO_MAX_VAXES][2][5] = {}, vC[DSO_MAX_VAXES][2][5] = {};
  for (auto& x : vbest)
    for (auto& y : x)
      for (float& z : y) z = 1e30f;
  std::memcpy(alt[0].G, c->G, sizeof(c->G));
  std::memcpy(alt[0].variant, c->variant, sizeof(c->variant));
  std::memcpy(alt[0].cps, c->cps, sizeof(c->cps));
  alt[1] = alt[0];
  for (const Pass& rp : reps) {
    if (err != cudaSuccess) break;
    Pass p = rp;
    p.u2 = -1;
    p.tb2 = -1;
    const int d = p.axis, SV = p.SV, which = SV == 1 ? 0 : 1;
    {
      const int L = kind_L(c, d, which);
      const long long lines = c->P / L;
      const int gmax = axis_pass_max_tile_lines(L, SV);
      bool any_whole = false;
      for (long long G = 1; G <= gmax && G <= lines; G *= 2)
        if ((SV * G * (L / 8)) % 32 == 0) any_whole = true;
      float best = 1e30f, best0 = 1e30f, bestN = 1e30f;
      int bestG = c->G[d][which], bestV = c->variant[d][which], bestC = c->cps[d][which];
      int bestG0 = bestG, bestGN = bestG, bestVN = -1, bestCN = 0;
      // DSO_VARIANT=v restricts the search to one kernel variant (testing)
      const char* fv = getenv("DSO_VARIANT");
      const int only = (fv && fv[0] >= '0' && fv[0] <= '4') ? fv[0] - '0' : -1;
      const bool both_tables = both[d][which];
      const int greg = c->vpart[d] == 1 ? 0 : axis_pass_reg_lines(L, SV);
      for (int var = 0; var < 5 && err == cudaSuccess; ++var) {
        if (only >= 0 && var != only) continue;
        if (var != 0 && var != 4 && c->prec == DSO_FP32) continue;  // variants 1-3 are FP64 only
        if (var == 3 && both_tables) continue;
        const bool reg = var == 4;
        if (reg && (greg == 0 || lines % greg)) continue;
        for (long long G = reg ? greg : 1; G <= (reg ? greg : gmax) && G <= lines && err == cudaSuccess; G *= 2) {
          if (!reg && any_whole && (SV * G * (L / 8)) % 32 != 0) continue;
          if (var == 1 && !axis_pass_pq_supported(L, SV, (int)G)) continue;
          if (var == 2 && !axis_pass_tma_supported(L, SV, (int)G)) continue;
          if (var == 3 && !axis_pass_tmap_supported(L, SV, (int)G)) continue;
          // persistent TMA: also the number of resident CTAs per SM
          static const int cps_try[4] = {0, 8, 4, 2};
          for (int ci = 0; ci < (var == 3 ? 4 : 1) && err == cudaSuccess; ++ci) {
            c->G[d][which] = (int)G;
            c->variant[d][which] = var;
            c->cps[d][which] = var == 3 ? cps_try[ci] : 0;
            err = run_pass(c, p);  // warm-up
            if (err == cudaErrorInvalidConfiguration) {  // does not fit (e.g. registers): not a candidate
              (void)cudaGetLastError();
              err = cudaSuccess;
              continue;
            }
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 10 && err == cudaSuccess; ++r) err = run_pass(c, p);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < best) {
              best = ms;
              bestG = (int)G;
              bestV = var;
              bestC = c->cps[d][which];
            }
            if (err == cudaSuccess && ms < vbest[d][which][var]) {
              vbest[d][which][var] = ms;
              vG[d][which][var] = (int)G;
              vC[d][which][var] = c->cps[d][which];
            }
            if (err == cudaSuccess && var == 0 && ms < best0) {
              best0 = ms;
              bestG0 = (int)G;
            }
            if (err == cudaSuccess && var != 0 && ms < bestN) {
              bestN = ms;
              bestGN = (int)G;
              bestVN = var;
              bestCN = c->cps[d][which];
            }
            const char* vb = getenv("DSO_TUNE_VERBOSE");
            if (vb && vb[0] == '1' && err == cudaSuccess)
              fprintf(stderr, "dso autotune: axis %d SV %d flags %d variant %d G %lld cps %d: %.2f us\n", d, SV,
                      p.flags, var, G, c->cps[d][which], ms * 1000.f / 10.f);
          }
        }
      }
      c->G[d][which] = bestG;
      c->variant[d][which] = bestV;
      c->cps[d][which] = bestC;
      // the kind's entries in the two other whole-step candidates
      alt[0].G[d][which] = best0 < 1e30f ? bestG0 : bestG;
      alt[0].variant[d][which] = best0 < 1e30f ? 0 : bestV;
      alt[0].cps[d][which] = best0 < 1e30f ? 0 : bestC;
      alt[1].G[d][which] = bestVN >= 0 ? bestGN : bestG;
      alt[1].variant[d][which] = bestVN >= 0 ? bestVN : bestV;
      alt[1].cps[d][which] = bestVN >= 0 ? bestCN : bestC;
    }
  }
  // Whole-step choice.  The passes are timed alone above, but a pass's cost
  // inside the step depends on its neighbours (programmatic dependent launch
  // overlaps the tail of one pass of the persistent, TMA or
  // register-resident variants with the start of the next, and is not used
  // next to the tile kernel; tables that stay in L2 across repeated
  // launches of one pass are evicted by the others).  So three candidate
  // plans -- the fastest variant of every kind, the tile kernel everywhere,
  // and the fastest of the other variants wherever one applies -- are timed
  // over host-launched middle steps, and the fastest is kept; then each kind,
  // in turn, tries its other variants that timed within 1.3x of its fastest
  // alone, kept where the whole middle step gets faster; then the plane pass.
  if (err == cudaSuccess && !getenv("DSO_VARIANT")) {
    const char* vb = getenv("DSO_TUNE_VERBOSE");
    const bool verbose = vb && vb[0] == '1';
    auto time_mid = [&](const std::vector<Pass>& mid, float& ms) {
      for (const Pass& p : mid)  // warm-up
        if (err == cudaSuccess) err = run_pass(c, p);
      if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3; ++r)
        for (const Pass& p : mid)
          if (err == cudaSuccess) err = run_pass(c, p);
      if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      return err == cudaSuccess;
    };
    TuneVal cand[3] = {};
    std::memcpy(cand[0].G, c->G, sizeof(c->G));
    std::memcpy(cand[0].variant, c->variant, sizeof(c->variant));
    std::memcpy(cand[0].cps, c->cps, sizeof(c->cps));
    cand[1] = alt[0];
    cand[2] = alt[1];
    const std::vector<Pass> mid = step_passes(c, false);
    float bestStep = 1e30f;
    int pick = 0;
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) {
      bool same = false;
      for (int j = 0; j < k; ++j)
        same = same || (std::memcmp(&cand[j], &cand[k], sizeof(TuneVal)) == 0);
      if (same) continue;
      std::memcpy(c->G, cand[k].G, sizeof(c->G));
      std::memcpy(c->variant, cand[k].variant, sizeof(c->variant));
      std::memcpy(c->cps, cand[k].cps, sizeof(c->cps));
      float ms = 0.f;
      if (!time_mid(mid, ms)) break;
      if (verbose)
        fprintf(stderr, "dso autotune: whole-step candidate %d: %.2f us per middle step\n", k, ms * 1000.f / 3.f);
      if (ms < bestStep) {
        bestStep = ms;
        pick = k;
      }
    }
    std::memcpy(c->G, cand[pick].G, sizeof(c->G));
    std::memcpy(c->variant, cand[pick].variant, sizeof(c->variant));
    std::memcpy(c->cps, cand[pick].cps, sizeof(c->cps));
    // coordinate descent over the kinds of the middle step
    std::vector<std::pair<int, int>> kinds;
    for (const Pass& p : mid) {
      const std::pair<int, int> k(p.axis, p.SV == 1 ? 0 : 1);
      if (!(p.flags & PASS_PLANE) && std::find(kinds.begin(), kinds.end(), k) == kinds.end()) kinds.push_back(k);
    }
    for (const auto& k : kinds) {
      const int d = k.first, w = k.second;
      float kbest = 1e30f;
      for (int v = 0; v < 5; ++v) kbest = std::min(kbest, vbest[d][w][v]);
      for (int v = 0; v < 5 && err == cudaSuccess; ++v) {
        if (v == c->variant[d][w] || vbest[d][w][v] >= 1e30f || vbest[d][w][v] > 1.3f * kbest) continue;
        const int g0 = c->G[d][w], v0 = c->variant[d][w], c0 = c->cps[d][w];
        c->G[d][w] = vG[d][w][v];
        c->variant[d][w] = v;
        c->cps[d][w] = vC[d][w][v];
        float ms = 0.f;
        if (!time_mid(mid, ms)) break;
        if (verbose)
          fprintf(stderr, "dso autotune: axis %d SV %s on variant %d: %.2f us per middle step\n", d,
                  w ? "S" : "1", v, ms * 1000.f / 3.f);
        if (ms < bestStep) {
          bestStep = ms;
        } else {
          c->G[d][w] = g0;
          c->variant[d][w] = v0;
          c->cps[d][w] = c0;
        }
      }
    }
    // DSO_PLANE_AUTO: the chosen plan's middle step once more with the plane
    // pass in place of the passes of axes 1 and 2
    if (err == cudaSuccess && c->plane_mode == DSO_PLANE_AUTO && !c->plane_on) {
      c->plane_on = true;
      if (plane_active(c)) {
        float ms = 0.f;
        const bool ok = time_mid(step_passes(c, false), ms);
        if (verbose && ok)
          fprintf(stderr, "dso autotune: with the plane pass: %.2f us per middle step\n", ms * 1000.f / 3.f);
        c->plane_on = ok && ms < bestStep;
      } else {
        c->plane_on = false;
      }
    }
  }
  c->psi = keep;
  c->launches = launches + (c->launches - launches);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CK(err);
  c->tuned = true;
  if (!getenv("DSO_VARIANT")) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    TuneVal v = {};
    std::memcpy(v.G, c->G, sizeof(v.G));
    std::memcpy(v.variant, c->variant, sizeof(v.variant));
    std::memcpy(v.cps, c->cps, sizeof(v.cps));
    v.plane = c->plane_on ? 1 : 0;
    g_tune_cache[tune_key(c)] = v;
  }
  return DSO_OK;
}

// Pass limits of small 1-D grids.  Unsplit, a 1-D grid of n <= 4096 points
// is one line: one CTA per job and surface set, so a small job runs on one
// SM (about 49 us per step for 1024 points and two surfaces, bound by that
// SM's FP64 pipe).  Split into two virtual axes (four-step), every pass has
// tens of lines and spreads over as many SMs, at the cost of a second pass
// and the twiddles.  For 1-D grids whose default plan is one line (S n <=
// 8192) the first propagation times a middle step under each candidate
// limit on a copy of psi and keeps the fastest.  The choice is cached per
// grid, surfaces, precision, elementary method and device -- not per batch
// size, so that a batch of such jobs and each job alone use the same layout
// and give bitwise the same result.  Skipped when the caller set the limits
// or forces a plan (DSO_PLAN).
using LimitsKey = std::tuple<int64_t, int, int, int, int>;
std::mutex g_limits_mu;
std::map<LimitsKey, std::pair<int, int>> g_limits_cache;

dso_status tune_limits(dso_ctx* c, double dt) {
  c->limits_tuned = true;
  if (c->limits_user || getenv("DSO_PLAN") || c->D != 1) return DSO_OK;
  if ((long long)c->S * c->n[0] > 8192) return DSO_OK;  // already split by default
  const char* env = getenv("DSO_AUTOTUNE");
  if (env && env[0] == '0') return DSO_OK;
  const LimitsKey key(c->n[0], c->S, c->prec, c->elementary, c->device);
  {
    std::lock_guard<std::mutex> lock(g_limits_mu);
    auto it = g_limits_cache.find(key);
    if (it != g_limits_cache.end()) {
      if (it->second.first != c->max_line || it->second.second != c->max_tile) {
        c->max_line = it->second.first;
        c->max_tile = it->second.second;
        return replan(c);
      }
      return DSO_OK;
    }
  }
  static const int cand[][2] = {{DSO_MAX_LINE, 8192}, {256, 512}, {128, 256}, {64, 128}, {32, 64}};
  const size_t bytes = (size_t)c->B * c->S * c->P * c->esz();
  if (!c->work) CK(cudaMalloc(&c->work, bytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  float best = 1e30f;
  int bl = c->max_line, bt = c->max_tile;
  for (const auto& cd : cand) {
    if (err != cudaSuccess) break;
    c->max_line = cd[0];
    c->max_tile = cd[1];
    if (replan(c) != DSO_OK) continue;  // the grid does not fit these limits
    dso_status st = ensure_tables(c, dt);
    if (st == DSO_OK) st = autotune_tiles(c);
    if (st != DSO_OK) {
      err = cudaErrorUnknown;
      break;
    }
    err = cudaMemcpyAsync(c->work, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream);
    void* keep = c->psi;
    c->psi = c->work;
    const std::vector<Pass> mid = step_passes(c, false);
    for (const Pass& p : mid)  // warm-up
      if (err == cudaSuccess) err = run_pass(c, p);
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 10 && err == cudaSuccess; ++r)
      for (const Pass& p : mid)
        if (err == cudaSuccess) err = run_pass(c, p);
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    c->psi = keep;
    if (err == cudaSuccess && ms < best) {
      best = ms;
      bl = cd[0];
      bt = cd[1];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CK(err);
  c->max_line = bl;
  c->max_tile = bt;
  dso_status st = replan(c);
  if (st != DSO_OK) return st;
  std::lock_guard<std::mutex> lock(g_limits_mu);
  g_limits_cache[key] = {bl, bt};
  return DSO_OK;
}

dso_status ensure_step_graph(dso_ctx* c) {
  if (c->step_exec) return DSO_OK;
  std::vector<Pass> passes = step_passes(c, false);
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  const int64_t before = c->launches;
  // The captured step is built without programmatic dependent launch: as
  // graph edges it measured slower (32^3 x 3, batch of 4, 512 replayed steps:
  // 1.83 s against 1.05 s), while host-launched passes gain from it.
  const int pdl = c->pdl;
  const char* pg = getenv("DSO_PDL_GRAPH");
  if (!(pg && pg[0] == '1')) c->pdl = 0;
  for (const Pass& p : passes) {
    err = run_pass(c, p);
    if (err != cudaSuccess) break;
  }
  c->pdl = pdl;
  c->launches = before;  // captured, not launched
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  if (err == cudaSuccess) err = e2;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&c->step_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  CK(err);
  c->step_exec_passes = (int)passes.size();
  return DSO_OK;
}

dso_status check_ready(dso_ctx* c) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (!c->have_grid) return fail(DSO_ESTATE, "grid not set");
  if (!c->have_V) return fail(DSO_ESTATE, "potential not loaded");
  if (!c->have_mass) return fail(DSO_ESTATE, "masses not set");
  if (!c->have_psi) return fail(DSO_ESTATE, "wavefunction not set");
  return DSO_OK;
}

dso_status ensure_coeffs(dso_ctx* c) {
  if (c->have_coeffs) return DSO_OK;
  c->coeffs = build_coefficients(c->order, c->scheme);
  c->have_coeffs = true;
  return DSO_OK;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" {

dso_status dso_create(dso_ctx** out, int device, int precision, void* cuda_stream) {
  if (!out) return fail(DSO_EINVAL, "out is null");
  *out = nullptr;
  if (precision != DSO_FP64 && precision != DSO_FP32) return fail(DSO_EINVAL, "precision must be DSO_FP64 or DSO_FP32");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(DSO_ECUDA, "no CUDA device");
  if (device < 0 || device >= ndev) return fail(DSO_EINVAL, "device index out of range");
  DeviceGuard g(device);
  if (!g.ok) return fail(DSO_ECUDA, "cudaSetDevice failed");
  dso_ctx* c = new (std::nothrow) dso_ctx();
  if (!c) return fail(DSO_ENOMEM, "host allocation failed");
  c->device = device;
  c->prec = precision;
  if (const char* e = getenv("DSO_PDL")) c->pdl = (e[0] == '0') ? 0 : 1;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(DSO_ECUDA, "stream creation failed");
    }
    c->own_stream = true;
  }
  *out = c;
  return DSO_OK;
}

void dso_destroy(dso_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_model(c);
  dfree(c->queue);
  dfree(c->err);
  for (auto& t : c->tw) dfree(t);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

dso_status dso_set_grid(dso_ctx* c, int D, const int64_t* n, const double* qmin, const double* qmax) {
  if (!c || !n || !qmin || !qmax) return fail(DSO_EINVAL, "null argument");
  if (D < 1 || D > DSO_MAX_DIM) return fail(DSO_EINVAL, "D must be 1..3");
  long long P = 1;
  for (int d = 0; d < D; ++d) {
    if (!is_pow2(n[d]) || n[d] < DSO_MIN_AXIS || n[d] > DSO_MAX_AXIS)
      return fail(DSO_EINVAL, "each n[d] must be a power of two in [8, 2^22]");
    if (!std::isfinite(qmin[d]) || !std::isfinite(qmax[d]) || !(qmax[d] > qmin[d]))
      return fail(DSO_EINVAL, "need finite qmin < qmax on every axis");
    P *= n[d];
  }
  if (P > DSO_MAX_POINTS) return fail(DSO_EINVAL, "the grid may have at most 2^30 points per surface");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_model(c);
  c->D = D;
  c->P = 1;
  for (int d = 0; d < DSO_MAX_DIM; ++d) {
    c->n[d] = d < D ? n[d] : 1;
    c->qmin[d] = d < D ? qmin[d] : 0.0;
    c->qmax[d] = d < D ? qmax[d] : 0.0;
    c->P *= c->n[d];
  }
  c->have_grid = true;
  c->have_mass = false;
  c->B = 1;
  c->limits_tuned = false;  // a new grid: chosen again at the first propagation
  if (!c->limits_user) {
    c->max_line = DSO_MAX_LINE;
    c->max_tile = 8192;
  }
  return DSO_OK;
}

dso_status dso_set_batch(dso_ctx* c, int B) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (!c->have_grid) return fail(DSO_ESTATE, "grid not set");
  if (B < 1 || B > (1 << 20)) return fail(DSO_EINVAL, "batch must be 1..2^20");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_model(c);
  c->B = B;
  c->limits_tuned = false;
  return DSO_OK;
}

dso_status dso_set_masses(dso_ctx* c, const double* m) {
  if (!c || !m) return fail(DSO_EINVAL, "null argument");
  if (!c->have_grid) return fail(DSO_ESTATE, "grid not set");
  for (int d = 0; d < c->D; ++d)
    if (!std::isfinite(m[d]) || !(m[d] > 0)) return fail(DSO_EINVAL, "masses must be finite and positive");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_tables(c);
  dfree(c->Tax);
  for (int d = 0; d < c->D; ++d) c->mass[d] = m[d];
  c->have_mass = true;
  return DSO_OK;
}

dso_status dso_load_potential(dso_ctx* c, int S, const double* V, int where) {
  if (!c || !V) return fail(DSO_EINVAL, "null argument");
  if (!c->have_grid) return fail(DSO_ESTATE, "grid not set");
  if (S < 2 || S > DSO_MAX_SURFACES) return fail(DSO_EINVAL, "S must be 2..4");
  if (where != DSO_HOST && where != DSO_DEVICE) return fail(DSO_EINVAL, "where must be DSO_HOST or DSO_DEVICE");
  const size_t count = (size_t)c->B * (S * (S + 1) / 2) * c->P;
  if (where == DSO_HOST) {
    for (size_t i = 0; i < count; ++i)
      if (!std::isfinite(V[i])) return fail(DSO_ENUMERIC, "potential has a non-finite value");
  }
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_model(c);
  c->S = S;
  c->limits_tuned = false;
  CK(cudaMalloc(&c->V, count * sizeof(double)));
  CK(cudaMemcpyAsync(c->V, V, count * sizeof(double), where == DSO_HOST ? cudaMemcpyHostToDevice
                                                                         : cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMalloc(&c->psi, (size_t)c->B * S * c->P * c->esz()));
  // Surface 0 uncoupled (V_0c = 0 on the whole grid for c > 0, in every job):
  // then U = exp(-i V t) is block diagonal and the V step skips U_0c.
  {
    std::vector<double> hv;
    const double* vh = V;
    if (where == DSO_DEVICE) {
      hv.resize(count);
      CK(cudaMemcpy(hv.data(), V, count * sizeof(double), cudaMemcpyDeviceToHost));
      vh = hv.data();
    }
    int dec = S > 2 ? 1 : 0;
    const size_t NPc = (size_t)S * (S + 1) / 2;
    for (int b = 0; b < c->B && dec; ++b)
      for (int k = 1; k < S && dec; ++k) {  // packed (0, k) sits at index k
        const double* row = vh + ((size_t)b * NPc + k) * c->P;
        for (long long g = 0; g < c->P; ++g)
          if (row[g] != 0.0) {
            dec = 0;
            break;
          }
      }
    c->dec0 = dec;
  }
  if (!c->queue) {
    CK(cudaMalloc(&c->queue, 2 * sizeof(unsigned)));
    CK(cudaMemsetAsync(c->queue, 0, 2 * sizeof(unsigned), c->stream));
  }
  if (!c->err) {
    CK(cudaMalloc(&c->err, 16 * sizeof(int)));
    CK(cudaMemsetAsync(c->err, 0, 16 * sizeof(int), c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  {
    const dso_status pst = replan(c);
    if (pst != DSO_OK) {
      drop_model(c);
      return pst;
    }
  }
  c->have_V = true;
  return DSO_OK;
}

dso_status dso_set_scheme(dso_ctx* c, int order, int scheme, int elementary, int prune) {
  if (!c) return fail(DSO_EINVAL, "null context");
  const bool first_order = elementary == DSO_VT || elementary == DSO_TV;
  if (first_order) {
    if (order != 1) return fail(DSO_EINVAL, "DSO_VT and DSO_TV are first-order: order must be 1");
    // TV (potential first) runs on the VTV machinery, VT (kinetic first) on TVT
    elementary = (elementary == DSO_TV) ? DSO_VTV : DSO_TVT;
    scheme = DSO_TRIPLE_JUMP;
  } else {
    if (order < 2 || order > 10 || order % 2) return fail(DSO_EINVAL, "order must be 2, 4, 6, 8 or 10");
    if (scheme != DSO_TRIPLE_JUMP && scheme != DSO_SUZUKI && scheme != DSO_OPTIMAL)
      return fail(DSO_EINVAL, "unknown scheme");
    if (scheme == DSO_OPTIMAL && order != 6 && order != 8)
      return fail(DSO_EINVAL, "the optimal compositions have orders 6 and 8");
    if (elementary != DSO_VTV && elementary != DSO_TVT)
      return fail(DSO_EINVAL, "elementary must be DSO_VTV, DSO_TVT, DSO_VT or DSO_TV");
  }
  if (prune != 1) return fail(DSO_EINVAL, "only pruned coefficients are part of this build");
  try {
    Coeffs cf = build_coefficients(order, scheme);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    drop_tables(c);
    c->coeffs = cf;
    c->order = order;
    c->scheme = scheme;
    if (c->elementary != elementary) c->tuned = false;  // other pass kinds
    c->elementary = elementary;
    c->have_coeffs = true;
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  return DSO_OK;
}

// Per-job squared norms sum |psi|^2 (no grid measure): block k of job b
// writes the sum of its grid-stride share to part[b * kNormBlocks + k]; the
// host adds the kNormBlocks values of a job in order, so the result is the
// same on every run.
constexpr int kNormBlocks = 64;
__global__ void norm_partial_kernel(const void* __restrict__ psi, long long per_job, int fp32, double* part) {
  __shared__ double red[256];
  const int b = blockIdx.y;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_job;
       i += (long long)gridDim.x * blockDim.x) {
    double re, im;
    if (fp32) {
      const float2 v = static_cast<const float2*>(psi)[b * per_job + i];
      re = v.x;
      im = v.y;
    } else {
      const double2 v = static_cast<const double2*>(psi)[b * per_job + i];
      re = v.x;
      im = v.y;
    }
    acc = fma(re, re, fma(im, im, acc));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[b * kNormBlocks + blockIdx.x] = red[0];
}

// Squared norms of every job's psi (synchronises the stream).
static dso_status job_norms(dso_ctx* c, std::vector<double>& out) {
  if (!c->norm_part || c->norm_part_cap < (size_t)c->B * kNormBlocks) {
    dfree(c->norm_part);
    CK(cudaMalloc(&c->norm_part, (size_t)c->B * kNormBlocks * sizeof(double)));
    c->norm_part_cap = (size_t)c->B * kNormBlocks;
  }
  norm_partial_kernel<<<dim3(kNormBlocks, c->B), 256, 0, c->stream>>>(c->psi, (long long)c->S * c->P,
                                                                       c->prec == DSO_FP32 ? 1 : 0, c->norm_part);
  CK(cudaGetLastError());
  c->launches += 1;
  std::vector<double> h((size_t)c->B * kNormBlocks);
  CK(cudaMemcpyAsync(h.data(), c->norm_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out.assign(c->B, 0.0);
  for (int b = 0; b < c->B; ++b)
    for (int k = 0; k < kNormBlocks; ++k) out[b] += h[(size_t)b * kNormBlocks + k];
  return DSO_OK;
}

// Per-job inner products sum conj(psi) phi (no grid measure): block k of job
// b writes the real and imaginary parts of its grid-stride share to
// part[(b * kNormBlocks + k) * 2 + {0, 1}]; the host adds them in order.
__global__ void inner_partial_kernel(const void* __restrict__ psi, const void* __restrict__ phi, long long per_job,
                                     int fp32, double* part) {
  __shared__ double red_re[256], red_im[256];
  const int b = blockIdx.y;
  double ar = 0.0, ai = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_job;
       i += (long long)gridDim.x * blockDim.x) {
    double xr, xi, yr, yi;
    if (fp32) {
      const float2 x = static_cast<const float2*>(psi)[b * per_job + i];
      const float2 y = static_cast<const float2*>(phi)[b * per_job + i];
      xr = x.x, xi = x.y, yr = y.x, yi = y.y;
    } else {
      const double2 x = static_cast<const double2*>(psi)[b * per_job + i];
      const double2 y = static_cast<const double2*>(phi)[b * per_job + i];
      xr = x.x, xi = x.y, yr = y.x, yi = y.y;
    }
    ar = fma(xr, yr, fma(xi, yi, ar));   // Re conj(x) y = xr yr + xi yi
    ai = fma(xr, yi, fma(-xi, yr, ai));  // Im conj(x) y = xr yi - xi yr
  }
  red_re[threadIdx.x] = ar;
  red_im[threadIdx.x] = ai;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red_re[threadIdx.x] += red_re[threadIdx.x + w];
      red_im[threadIdx.x] += red_im[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[(b * kNormBlocks + blockIdx.x) * 2] = red_re[0];
    part[(b * kNormBlocks + blockIdx.x) * 2 + 1] = red_im[0];
  }
}

// Largest density |psi_s(q)|^2 of every (job, surface) row: block k of row r
// writes its (density, first index of it, re, im) to part[(r * kNormBlocks + k)
// * 4 + {0..3}] (the index as a double: exact below 2^53).  Ties keep the
// smallest index, so the host's in-order reduction gives the first maximum in
// storage order.
__global__ void density_max_kernel(const void* __restrict__ psi, long long P, int fp32, double* part) {
  __shared__ double rd[256], ri[256];
  __shared__ long long rx[256];
  const long long row = blockIdx.y;
  double best = -1.0, br = 0.0, bi = 0.0;
  long long bx = -1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    double re, im;
    if (fp32) {
      const float2 v = static_cast<const float2*>(psi)[row * P + i];
      re = v.x, im = v.y;
    } else {
      const double2 v = static_cast<const double2*>(psi)[row * P + i];
      re = v.x, im = v.y;
    }
    const double d = re * re + im * im;
    if (d > best) {  // i grows: a later equal value never replaces
      best = d, bx = i, br = re, bi = im;
    }
  }
  rd[threadIdx.x] = best;
  rx[threadIdx.x] = bx;
  ri[threadIdx.x] = br;
  __syncthreads();
  __shared__ double rim[256];
  rim[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const int o = threadIdx.x + w;
      const bool take = rd[o] > rd[threadIdx.x] ||
                        (rd[o] == rd[threadIdx.x] && rx[o] >= 0 && (rx[threadIdx.x] < 0 || rx[o] < rx[threadIdx.x]));
      if (take) {
        rd[threadIdx.x] = rd[o];
        rx[threadIdx.x] = rx[o];
        ri[threadIdx.x] = ri[o];
        rim[threadIdx.x] = rim[o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* out = part + (row * kNormBlocks + blockIdx.x) * 4;
    out[0] = rd[0];
    out[1] = (double)rx[0];
    out[2] = ri[0];
    out[3] = rim[0];
  }
}

// A user composition: 1..4096 finite nonzero elementary coefficients,
// symmetric, summing to one.
static dso_status check_gammas(int m, const double* gamma, std::vector<long double>& g) {
  if (m < 1 || m > 4096 || !gamma) return fail(DSO_EINVAL, "need 1..4096 composition coefficients");
  long double sum = 0.0L;
  double big = 0.0;
  g.assign(m, 0.0L);
  for (int k = 0; k < m; ++k) {
    if (!std::isfinite(gamma[k]) || gamma[k] == 0.0)
      return fail(DSO_EINVAL, "composition coefficients must be finite and nonzero");
    g[k] = gamma[k];
    sum += g[k];
    big = std::fmax(big, std::fabs(gamma[k]));
  }
  if (fabsl(sum - 1.0L) > 1e-13L) return fail(DSO_EINVAL, "composition coefficients must sum to 1");
  for (int k = 0; k < m; ++k)
    if (std::fabs(gamma[k] - gamma[m - 1 - k]) > 1e-14 * big)
      return fail(DSO_EINVAL, "the composition must be symmetric (gamma_k = gamma_{m+1-k})");
  return DSO_OK;
}

// Finite check of a staged copy of psi on the device: a word whose exponent
// bits are all ones (Inf or NaN) sets *flag.  n counts 8-byte words (FP64
// components) or 4-byte words (FP32).
__global__ void nonfinite_flag_kernel(const void* __restrict__ p, long long n, int fp32, int* flag) {
  int bad = 0;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
  if (fp32) {
    const unsigned* u = static_cast<const unsigned*>(p);
    for (long long i = i0; i < n; i += step) bad |= (u[i] & 0x7f800000u) == 0x7f800000u;
  } else {
    const unsigned long long* u = static_cast<const unsigned long long*>(p);
    for (long long i = i0; i < n; i += step) bad |= (u[i] & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

dso_status dso_set_composition(dso_ctx* c, int m, const double* gamma, int elementary) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (elementary != DSO_VTV && elementary != DSO_TVT) return fail(DSO_EINVAL, "elementary must be DSO_VTV or DSO_TVT");
  std::vector<long double> g;
  dso_status st = check_gammas(m, gamma, g);
  if (st != DSO_OK) return st;
  try {
    Coeffs cf = coefficients_from_gammas(g);
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    drop_tables(c);
    c->coeffs = cf;
    c->order = 0;  // a user composition
    c->scheme = -1;
    if (c->elementary != elementary) c->tuned = false;
    c->elementary = elementary;
    c->have_coeffs = true;
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  return DSO_OK;
}

dso_status dso_set_wait_probe(dso_ctx* c, int polls) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (polls < 0) return fail(DSO_EINVAL, "polls must be >= 0");
  c->wait_probe = polls;
  drop_graph(c);  // the captured step carries the launch arguments
  return DSO_OK;
}

dso_status dso_psi_device_pointer(dso_ctx* c, void** out) {
  if (!c || !out) return fail(DSO_EINVAL, "null argument");
  if (!c->psi) return fail(DSO_ESTATE, "load the potential first (it allocates psi)");
  *out = c->psi;
  return DSO_OK;
}

dso_status dso_set_norm_check(dso_ctx* c, double tol) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (!std::isfinite(tol) || tol < 0.0) return fail(DSO_EINVAL, "tol must be finite and >= 0");
  c->norm_tol = tol;
  c->norm_ref.clear();  // taken again from the current psi at the next check
  return DSO_OK;
}

dso_status dso_composition_coefficients(int m, const double* gamma, int* n_a, int* n_b, double* a, double* b,
                                        int* ia, int* ib, int* n_a_unq, int* n_b_unq) {
  std::vector<long double> g;
  dso_status st = check_gammas(m, gamma, g);
  if (st != DSO_OK) return st;
  Coeffs cf = coefficients_from_gammas(g);
  if (n_a) *n_a = (int)cf.a.size();
  if (n_b) *n_b = (int)cf.b.size();
  if (n_a_unq) *n_a_unq = (int)cf.a_unq.size();
  if (n_b_unq) *n_b_unq = (int)cf.b_unq.size();
  if (a) std::memcpy(a, cf.a.data(), cf.a.size() * sizeof(double));
  if (b) std::memcpy(b, cf.b.data(), cf.b.size() * sizeof(double));
  if (ia) std::memcpy(ia, cf.ia.data(), cf.ia.size() * sizeof(int));
  if (ib) std::memcpy(ib, cf.ib.data(), cf.ib.size() * sizeof(int));
  return DSO_OK;
}

dso_status dso_set_psi(dso_ctx* c, const void* psi, int where) {
  if (!c || !psi) return fail(DSO_EINVAL, "null argument");
  if (!c->have_V) return fail(DSO_ESTATE, "load the potential first (it fixes S)");
  if (where != DSO_HOST && where != DSO_DEVICE) return fail(DSO_EINVAL, "where must be DSO_HOST or DSO_DEVICE");
  const size_t bytes = (size_t)c->B * c->S * c->P * c->esz();
  DeviceGuard g(c->device);
  if (where == DSO_HOST) {
    // Stage the host data in the work buffer, check it there (a few
    // microseconds on the device instead of a pass over the host array), and
    // only then copy it into psi, so a rejected input leaves psi unchanged.
    if (!c->work) CK(cudaMalloc(&c->work, bytes));
    int* flag = c->err + 15;
    CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    CK(cudaMemcpyAsync(c->work, psi, bytes, cudaMemcpyHostToDevice, c->stream));
    const long long words = 2LL * c->B * c->S * c->P;
    const unsigned blocks = (unsigned)std::min<long long>((words + 255) / 256, 4096);
    nonfinite_flag_kernel<<<blocks, 256, 0, c->stream>>>(c->work, words, c->prec == DSO_FP32 ? 1 : 0, flag);
    CK(cudaGetLastError());
    c->launches += 1;
    int hflag = 0;
    CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hflag) return fail(DSO_ENUMERIC, "psi has a non-finite value");
    CK(cudaMemcpyAsync(c->psi, c->work, bytes, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(cudaMemcpyAsync(c->psi, psi, bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  c->have_psi = true;
  c->norm_ref.clear();  // a new state: the norm monitor takes its reference again
  return DSO_OK;
}

dso_status dso_propagate(dso_ctx* c, double t, double dt) {
  NvtxRange nvtx("dso_propagate");
  dso_status st = check_ready(c);
  if (st != DSO_OK) return st;
  if (!std::isfinite(t) || !std::isfinite(dt) || dt == 0.0) return fail(DSO_EINVAL, "t and dt must be finite, dt != 0");
  const double ratio = t / dt;
  const double nr = std::round(ratio);
  if (nr < 0 || std::fabs(ratio - nr) > 1e-9 * std::fmax(1.0, std::fabs(ratio)))
    return fail(DSO_EINVAL, "t / dt must be a non-negative integer");
  const long long nsteps = (long long)nr;
  if (nsteps == 0) return DSO_OK;
  DeviceGuard g(c->device);
  try {
    st = ensure_coeffs(c);
    if (st != DSO_OK) return st;
    if (!c->limits_tuned) {
      st = tune_limits(c, dt);
      if (st != DSO_OK) return st;
    }
    st = ensure_tables(c, dt);
    if (st != DSO_OK) return st;
    if (!c->tuned) {
      drop_graph(c);
      st = autotune_tiles(c);
      if (st != DSO_OK) return st;
    }
    if (c->norm_tol > 0.0 && c->norm_ref.empty()) {
      st = job_norms(c, c->norm_ref);
      if (st != DSO_OK) return st;
    }
    for (const Pass& p : step_passes(c, true)) CK(run_pass(c, p));
    if (nsteps > 1) {
      const bool capturable = c->stream != nullptr && c->stream != cudaStreamLegacy && c->stream != cudaStreamPerThread;
      if (capturable) {
        st = ensure_step_graph(c);
        if (st != DSO_OK) return st;
        for (long long s = 1; s < nsteps; ++s) {
          CK(cudaGraphLaunch(c->step_exec, c->stream));
          c->launches += c->step_exec_passes;
        }
      } else {
        const std::vector<Pass> mid = step_passes(c, false);
        for (long long s = 1; s < nsteps; ++s)
          for (const Pass& p : mid) CK(run_pass(c, p));
      }
    }
    for (const Pass& p : final_passes(c)) CK(run_pass(c, p));
    if (c->norm_tol > 0.0) {  // the propagation is unitary: the norm may move by round-off only
      std::vector<double> now;
      st = job_norms(c, now);
      if (st != DSO_OK) return st;
      for (int b = 0; b < c->B; ++b) {
        const double ref = c->norm_ref[b], drift = std::fabs(std::sqrt(now[b]) - std::sqrt(ref));
        if (!(drift <= c->norm_tol * std::sqrt(ref)))
          return fail(DSO_ENUMERIC, "norm of job " + std::to_string(b) + " drifted by " + std::to_string(drift) +
                                        " (relative tolerance " + std::to_string(c->norm_tol) + ")");
      }
    }
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  return DSO_OK;
}

// A kernel whose bounded wait gave up leaves a code in c->err; report it at
// the next synchronising call.
static dso_status check_device_flag(dso_ctx* c) {
  if (!c->err) return DSO_OK;
  int h[16] = {};
  CK(cudaMemcpyAsync(h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h[0] != 0) {
    CK(cudaMemsetAsync(c->err, 0, sizeof(h), c->stream));
    std::string ctx_info;
    if (h[1])  // bounds-checked debug build: context of the first bad access
      for (int i = 2; i < 10; ++i) ctx_info += " " + std::to_string(h[i]);
    if (h[0] >= 100)
      return fail(DSO_ECUDA, "bounds check failed in an axis pass (code " + std::to_string(h[0]) + ")" + ctx_info);
    if (h[0] == 5)
      return fail(DSO_ETIMEOUT, "the diagnostic bounded wait (dso_set_wait_probe) gave up, as it must (code 5)");
    return fail(DSO_ETIMEOUT, "a kernel's bounded wait for its tile copy gave up (code " + std::to_string(h[0]) + ")");
  }
  return DSO_OK;
}

dso_status dso_get_psi(dso_ctx* c, void* out, int where) {
  if (!c || !out) return fail(DSO_EINVAL, "null argument");
  if (!c->have_psi) return fail(DSO_ESTATE, "wavefunction not set");
  if (where != DSO_HOST && where != DSO_DEVICE) return fail(DSO_EINVAL, "where must be DSO_HOST or DSO_DEVICE");
  DeviceGuard g(c->device);
  const size_t bytes = (size_t)c->B * c->S * c->P * c->esz();
  CK(cudaMemcpyAsync(out, c->psi, bytes, where == DSO_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     c->stream));
  // the error flags come back after the copy, under the same synchronisation
  if (where == DSO_HOST) return check_device_flag(c);
  return DSO_OK;
}

dso_status dso_observables(dso_ctx* c, double* norm, double* energy, double* pops) {
  NvtxRange nvtx("dso_observables");
  dso_status st = check_ready(c);
  if (st != DSO_OK) return st;
  DeviceGuard g(c->device);
  st = ensure_twiddles(c);
  if (st != DSO_OK) return st;
  if (!c->Tax) {
    std::vector<double> h;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int d = 0; d < c->D; ++d)
      for (int64_t k = 0; k < c->n[d]; ++k) {
        const int64_t kk = (k < c->n[d] / 2) ? k : k - c->n[d];
        const long double p = two_pi * (long double)kk / ((long double)c->qmax[d] - (long double)c->qmin[d]);
        h.push_back((double)(p * p / (2.0L * (long double)c->mass[d])));
      }
    CK(cudaMalloc(&c->Tax, h.size() * sizeof(double)));
    CK(cudaMemcpy(c->Tax, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (!c->work) CK(cudaMalloc(&c->work, (size_t)c->B * c->S * c->P * c->esz()));
  if (!c->partials) CK(cudaMalloc(&c->partials, (size_t)obs_partial_blocks() * DSO_OBS_COLS * sizeof(double)));
  if (!c->obs_out) CK(cudaMalloc(&c->obs_out, (size_t)c->B * DSO_OBS_COLS * sizeof(double)));
  // momentum representation of a copy: forward FFT along every axis
  CK(cudaMemcpyAsync(c->work, c->psi, (size_t)c->B * c->S * c->P * c->esz(), cudaMemcpyDeviceToDevice,
                     c->stream));
  void* keep = c->psi;
  c->psi = c->work;
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < c->Dv && e == cudaSuccess; ++d) e = run_pass(c, mkpass(d, 1, PASS_FWD));
  c->psi = keep;
  CK(e);
  const int NPV = c->S * (c->S + 1) / 2;
  for (int b = 0; b < c->B; ++b) {
    ObsArgs a;
    a.psi = at(c->psi, (size_t)b * c->S * c->P, c->esz());
    a.psik = at(c->work, (size_t)b * c->S * c->P, c->esz());
    a.fp32 = c->prec == DSO_FP32 ? 1 : 0;
    a.V = c->V + (size_t)b * NPV * c->P;
    a.Tax = c->Tax;
    a.vl = vlayout(c);
    a.S = c->S;
    a.P = c->P;
    CK(launch_observables(a, c->partials, c->obs_out + (size_t)b * DSO_OBS_COLS, c->stream));
    c->launches += 2;
  }
  std::vector<double> h((size_t)c->B * DSO_OBS_COLS);
  CK(cudaMemcpyAsync(h.data(), c->obs_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double dV = 1.0;
  for (int d = 0; d < c->D; ++d) dV *= (c->qmax[d] - c->qmin[d]) / (double)c->n[d];
  bool finite = true;
  for (int b = 0; b < c->B; ++b) {
    const double* hb = h.data() + (size_t)b * DSO_OBS_COLS;
    double tot = 0.0;
    for (int s = 0; s < c->S; ++s) {
      if (pops) pops[(size_t)b * c->S + s] = hb[s] * dV;
      tot += hb[s];
    }
    if (norm) norm[b] = std::sqrt(tot * dV);
    if (energy) energy[b] = hb[c->S] * dV + hb[c->S + 1] * dV / (double)c->P;
    finite = finite && std::isfinite(tot) && std::isfinite(hb[c->S]) && std::isfinite(hb[c->S + 1]);
  }
  if (!finite) return fail(DSO_ENUMERIC, "non-finite observable");
  return DSO_OK;
}

dso_status dso_inner(dso_ctx* c, const void* phi, int where, double* re, double* im) {
  NvtxRange nvtx("dso_inner");
  if (!c || !phi) return fail(DSO_EINVAL, "null argument");
  if (!c->have_psi) return fail(DSO_ESTATE, "wavefunction not set");
  if (where != DSO_HOST && where != DSO_DEVICE) return fail(DSO_EINVAL, "where must be DSO_HOST or DSO_DEVICE");
  DeviceGuard g(c->device);
  const size_t bytes = (size_t)c->B * c->S * c->P * c->esz();
  const void* dphi = phi;
  if (where == DSO_HOST) {  // staged in the work buffer
    if (!c->work) CK(cudaMalloc(&c->work, bytes));
    CK(cudaMemcpyAsync(c->work, phi, bytes, cudaMemcpyHostToDevice, c->stream));
    dphi = c->work;
  }
  if (!c->norm_part || c->norm_part_cap < (size_t)c->B * kNormBlocks * 4) {
    dfree(c->norm_part);
    CK(cudaMalloc(&c->norm_part, (size_t)c->B * kNormBlocks * 4 * sizeof(double)));
    c->norm_part_cap = (size_t)c->B * kNormBlocks * 4;
  }
  inner_partial_kernel<<<dim3(kNormBlocks, c->B), 256, 0, c->stream>>>(c->psi, dphi, (long long)c->S * c->P,
                                                                        c->prec == DSO_FP32 ? 1 : 0, c->norm_part);
  CK(cudaGetLastError());
  c->launches += 1;
  std::vector<double> h((size_t)c->B * kNormBlocks * 2);
  CK(cudaMemcpyAsync(h.data(), c->norm_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double dV = 1.0;
  for (int d = 0; d < c->D; ++d) dV *= (c->qmax[d] - c->qmin[d]) / (double)c->n[d];
  for (int b = 0; b < c->B; ++b) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < kNormBlocks; ++k) {
      sr += h[((size_t)b * kNormBlocks + k) * 2];
      si += h[((size_t)b * kNormBlocks + k) * 2 + 1];
    }
    if (re) re[b] = sr * dV;
    if (im) im[b] = si * dV;
  }
  return DSO_OK;
}

dso_status dso_phase_at_density_maximum(dso_ctx* c, int64_t* index, double* phase) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (!c->have_psi) return fail(DSO_ESTATE, "wavefunction not set");
  DeviceGuard g(c->device);
  const long long rows = (long long)c->B * c->S;
  if (rows > 65535) return fail(DSO_EINVAL, "at most 65535 job surfaces");
  if (!c->norm_part || c->norm_part_cap < (size_t)rows * kNormBlocks * 4) {
    dfree(c->norm_part);
    CK(cudaMalloc(&c->norm_part, (size_t)rows * kNormBlocks * 4 * sizeof(double)));
    c->norm_part_cap = (size_t)rows * kNormBlocks * 4;
  }
  density_max_kernel<<<dim3(kNormBlocks, (unsigned)rows), 256, 0, c->stream>>>(c->psi, c->P,
                                                                             c->prec == DSO_FP32 ? 1 : 0,
                                                                             c->norm_part);
  CK(cudaGetLastError());
  c->launches += 1;
  std::vector<double> h((size_t)rows * kNormBlocks * 4);
  CK(cudaMemcpyAsync(h.data(), c->norm_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (long long r = 0; r < rows; ++r) {
    double best = -1.0, br = 0.0, bi = 0.0;
    long long bx = -1;
    for (int k = 0; k < kNormBlocks; ++k) {
      const double* p = &h[((size_t)r * kNormBlocks + k) * 4];
      const long long x = (long long)p[1];
      if (x < 0) continue;
      if (p[0] > best || (p[0] == best && x < bx)) {
        best = p[0], bx = x, br = p[2], bi = p[3];
      }
    }
    if (index) index[r] = bx;
    if (phase) phase[r] = std::atan2(bi, br);
  }
  return DSO_OK;
}

dso_status dso_scheme_coefficients(int order, int scheme, int* n_a, int* n_b, double* a, double* b, int* ia,
                                   int* ib, int* n_a_unq, int* n_b_unq) {
  Coeffs cf;
  try {
    cf = build_coefficients(order, scheme);
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  if (n_a) *n_a = (int)cf.a.size();
  if (n_b) *n_b = (int)cf.b.size();
  if (n_a_unq) *n_a_unq = (int)cf.a_unq.size();
  if (n_b_unq) *n_b_unq = (int)cf.b_unq.size();
  if (a) std::memcpy(a, cf.a.data(), cf.a.size() * sizeof(double));
  if (b) std::memcpy(b, cf.b.data(), cf.b.size() * sizeof(double));
  if (ia) std::memcpy(ia, cf.ia.data(), cf.ia.size() * sizeof(int));
  if (ib) std::memcpy(ib, cf.ib.data(), cf.ib.size() * sizeof(int));
  return DSO_OK;
}

dso_status dso_profile_steps(dso_ctx* c, double dt, int nsteps, int max_kinds, int* n_kinds, int* axis, int* flags,
                             int* surfaces, int* launches_per_step, double* avg_ms, int* tile_lines, int* variant) {
  dso_status st = check_ready(c);
  if (st != DSO_OK) return st;
  if (!std::isfinite(dt) || dt == 0.0 || nsteps < 1) return fail(DSO_EINVAL, "need finite dt != 0 and nsteps >= 1");
  DeviceGuard g(c->device);
  try {
    st = ensure_coeffs(c);
    if (st != DSO_OK) return st;
    st = ensure_tables(c, dt);
    if (st != DSO_OK) return st;
    if (!c->tuned) {
      drop_graph(c);
      st = autotune_tiles(c);
      if (st != DSO_OK) return st;
    }
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  const std::vector<Pass> passes = step_passes(c, false);
  struct Kind {
    int axis, flags, sv, count;
    double ms;
  };
  std::vector<Kind> kinds;
  std::vector<int> kind_of(passes.size());
  for (size_t i = 0; i < passes.size(); ++i) {
    const Pass& p = passes[i];
    const int f = p.flags | (p.u1 >= 0 ? 256 : 0) | (p.u2 >= 0 ? 512 : 0) | (p.tb2 >= 0 ? 1024 : 0);
    int k = -1;
    for (size_t j = 0; j < kinds.size(); ++j)
      if (kinds[j].axis == p.axis && kinds[j].flags == f && kinds[j].sv == p.SV) k = (int)j;
    if (k < 0) {
      kinds.push_back(Kind{p.axis, f, p.SV, 0, 0.0});
      k = (int)kinds.size() - 1;
    }
    kinds[k].count += 1;
    kind_of[i] = k;
  }
  std::vector<cudaEvent_t> ev(2 * passes.size(), nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
    for (size_t i = 0; i < passes.size() && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[2 * i], c->stream);
      if (e == cudaSuccess) e = run_pass(c, passes[i]);
      if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    for (size_t i = 0; i < passes.size() && e == cudaSuccess; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      kinds[kind_of[i]].ms += ms;
    }
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  CK(e);
  if (n_kinds) *n_kinds = (int)kinds.size();
  for (int k = 0; k < (int)kinds.size() && k < max_kinds; ++k) {
    if (axis) axis[k] = kinds[k].axis;
    if (flags) flags[k] = kinds[k].flags;
    if (surfaces) surfaces[k] = kinds[k].sv;
    if (launches_per_step) launches_per_step[k] = kinds[k].count;
    if (avg_ms) avg_ms[k] = kinds[k].ms / ((double)kinds[k].count * nsteps);
    const int which = kinds[k].sv == 1 ? 0 : 1;
    if (tile_lines) tile_lines[k] = c->G[kinds[k].axis][which];
    if (variant) variant[k] = c->variant[kinds[k].axis][which];
  }
  return DSO_OK;
}

int dso_busy(const dso_ctx* c) {
  if (!c) return fail(DSO_EINVAL, "null context");
  DeviceGuard g(c->device);
  const cudaError_t e = cudaStreamQuery(c->stream);
  if (e == cudaSuccess) return 0;
  if (e == cudaErrorNotReady) return 1;
  return fail(DSO_ECUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
}

int64_t dso_launch_count(const dso_ctx* c) { return c ? c->launches : 0; }

int dso_tuned_plan(const dso_ctx* c, char* out, int cap) {
  if (!c || !out || cap < 1) return fail(DSO_EINVAL, "dso_tuned_plan: null argument");
  std::string s;
  for (int d = 0; d < c->Dv; ++d)
    for (int w = 0; w < 2; ++w) {
      char e[64];
      snprintf(e, sizeof(e), "%d,%d,%d,%d,%d;", d, w, c->variant[d][w], c->G[d][w], c->cps[d][w]);
      s += e;
    }
  if (plane_active(c)) s += "plane;";
  if ((int)s.size() + 1 > cap) return fail(DSO_EINVAL, "dso_tuned_plan: buffer too small");
  std::memcpy(out, s.c_str(), s.size() + 1);
  return (int)s.size();
}

dso_status dso_set_boundary_merge(dso_ctx* c, int merged) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (merged != 0 && merged != 1) return fail(DSO_EINVAL, "merged must be 0 or 1");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_tables(c);
  c->boundary_merged = merged;
  c->tuned = false;  // other pass kinds
  return DSO_OK;
}

dso_status dso_set_kinetic_mode(dso_ctx* c, int mode) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (mode != DSO_KINETIC_AUTO && mode != DSO_KINETIC_JOINT && mode != DSO_KINETIC_AXES)
    return fail(DSO_EINVAL, "mode must be DSO_KINETIC_AUTO, DSO_KINETIC_JOINT or DSO_KINETIC_AXES");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_tables(c);
  c->kin_mode = mode;
  c->tuned = false;  // other pass kinds
  return DSO_OK;
}

dso_status dso_set_operator_mode(dso_ctx* c, int mode) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (mode != DSO_OPERATORS_AUTO && mode != DSO_OPERATORS_TABLES && mode != DSO_OPERATORS_ON_THE_FLY)
    return fail(DSO_EINVAL, "mode must be DSO_OPERATORS_AUTO, DSO_OPERATORS_TABLES or DSO_OPERATORS_ON_THE_FLY");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_tables(c);
  c->op_mode = mode;
  c->tuned = false;  // the passes' costs change
  return DSO_OK;
}

int dso_operators_on_the_fly(const dso_ctx* c) {
  if (!c) return fail(DSO_EINVAL, "null context");
  return c->tables_valid && c->otf ? 1 : 0;
}

dso_status dso_set_plane_pass(dso_ctx* c, int mode) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (mode != DSO_PLANE_AUTO && mode != DSO_PLANE_OFF && mode != DSO_PLANE_ON)
    return fail(DSO_EINVAL, "mode must be DSO_PLANE_AUTO, DSO_PLANE_OFF or DSO_PLANE_ON");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  drop_graph(c);
  c->plane_mode = mode;
  c->plane_on = false;
  c->tuned = false;  // other pass list
  return DSO_OK;
}

dso_status dso_set_pass_limits(dso_ctx* c, int max_line, int max_tile) {
  if (!c) return fail(DSO_EINVAL, "null context");
  if (max_line < 8 || max_line > DSO_MAX_LINE || (max_line & (max_line - 1)) || max_tile < 16 || max_tile > 8192 ||
      (max_tile & (max_tile - 1)))
    return fail(DSO_EINVAL, "max_line must be a power of two in [8, 4096] and max_tile one in [16, 8192]");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  const int ol = c->max_line, ot = c->max_tile;
  c->max_line = max_line;
  c->max_tile = max_tile;
  c->limits_user = true;
  if (c->have_V) {  // S is known: plan again (psi is in the position representation: unaffected)
    const dso_status st = replan(c);
    if (st != DSO_OK) {
      c->max_line = ol;
      c->max_tile = ot;
      const dso_status back = replan(c);
      (void)back;
      return st;
    }
  }
  return DSO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch slots: many jobs (contexts) with uneven grids advance by one composed
// step per persistent launch of the work-list kernel (batch.cu).
// ---------------------------------------------------------------------------

namespace {

constexpr int kBatchMaxLine = 1024;  // batch tiles hold at most 2048 amplitudes:
constexpr int kBatchMaxTile = 2048;  // lines of <= 1024 points, S n1 <= 2048 on axis 0

struct BatchSlot {
  dso_ctx* ctx = nullptr;
  double dt = 0.0;
  long long steps_total = 0, steps_done = 0;
  bool live = false;
  std::vector<BatchPass> first, mid, fin;  // pass lists of a first, a middle and the final step
};

}  // namespace

struct dso_batch {
  int device = 0;
  int prec = DSO_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<BatchSlot> slots;
  // device work list of the next launch
  BatchPass* d_pass = nullptr;
  size_t pass_cap = 0;
  BatchSeg* d_seg = nullptr;
  size_t seg_cap = 0;
  unsigned* d_done = nullptr;  // per-segment completion counters
  size_t done_cap = 0;
  unsigned long long* d_head = nullptr;
  int* d_err = nullptr;
  std::vector<BatchPass> h_pass;  // host copies of the last launch's list (kept until it completes)
  std::vector<BatchSeg> h_seg;
  int64_t launches = 0;
};

namespace {

dso_status batch_reserve(dso_batch* b, size_t npass, size_t nseg) {
  if (npass > b->pass_cap) {
    dfree(b->d_pass);
    b->pass_cap = std::max(npass, 2 * b->pass_cap);
    CK(cudaMalloc(&b->d_pass, b->pass_cap * sizeof(BatchPass)));
  }
  if (nseg > b->seg_cap) {
    dfree(b->d_seg);
    b->seg_cap = std::max(nseg, 2 * b->seg_cap);
    CK(cudaMalloc(&b->d_seg, b->seg_cap * sizeof(BatchSeg)));
  }
  if (nseg > b->done_cap) {
    dfree(b->d_done);
    b->done_cap = std::max(nseg, 2 * b->done_cap);
    CK(cudaMalloc(&b->d_done, b->done_cap * sizeof(unsigned)));
  }
  return DSO_OK;
}

// The batch's tile line count for pass kinds of line length L staging SV
// surfaces: the largest power of two G with SV G L <= 2048 amplitudes (one
// 8-value slot per thread of a 256-thread CTA), at most the lines per surface.
int batch_G(const dso_ctx* c, int L, int SV) {
  const long long lines = c->P / L;
  long long G = 1;
  while (G * 2 <= lines && (long long)SV * G * 2 * L <= batch_max_tile_amplitudes()) G *= 2;
  return (int)G;
}

dso_status batch_list(dso_ctx* c, const std::vector<Pass>& passes, std::vector<BatchPass>& out) {
  out.clear();
  for (const Pass& p : passes) {
    if (p.flags & PASS_PLANE) return fail(DSO_EINVAL, "internal: the plane pass in a batch slot");
    BatchPass bp{};
    long long ntiles = 0;
    const cudaError_t e = build_pass_args(c, p, bp.a, ntiles);
    if (e != cudaSuccess) return fail(DSO_EINVAL, std::string("batch pass arguments: ") + cudaGetErrorString(e));
    bp.L = (int)c->nv[p.axis];
    bp.log2L = ilog2(bp.L);
    bp.SV = p.SV;
    bp.ntiles = ntiles;
    if ((long long)bp.SV * bp.a.G * bp.L > batch_max_tile_amplitudes())
      return fail(DSO_EINVAL, "internal: a batch tile exceeds the kernel's tile");
    out.push_back(bp);
  }
  return DSO_OK;
}

}  // namespace

extern "C" {

dso_status dso_batch_create(dso_batch** out, int device, int precision, void* cuda_stream) {
  if (!out) return fail(DSO_EINVAL, "out is null");
  *out = nullptr;
  if (precision != DSO_FP64 && precision != DSO_FP32) return fail(DSO_EINVAL, "precision must be DSO_FP64 or DSO_FP32");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(DSO_ECUDA, "no CUDA device");
  if (device < 0 || device >= ndev) return fail(DSO_EINVAL, "device index out of range");
  DeviceGuard g(device);
  dso_batch* b = new (std::nothrow) dso_batch();
  if (!b) return fail(DSO_ENOMEM, "host allocation failed");
  b->device = device;
  b->prec = precision;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail(DSO_ECUDA, "stream creation failed");
  } else {
    b->own_stream = true;
  }
  if (cudaMalloc(&b->d_head, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream)) {
    dfree(b->d_head);
    dfree(b->d_err);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return fail(DSO_ENOMEM, "device allocation failed");
  }
  *out = b;
  return DSO_OK;
}

void dso_batch_destroy(dso_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  dfree(b->d_pass);
  dfree(b->d_seg);
  dfree(b->d_done);
  dfree(b->d_head);
  dfree(b->d_err);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

dso_status dso_batch_add(dso_batch* b, dso_ctx* c, double t, double dt, int* slot) {
  NvtxRange nvtx("dso_batch_add");
  if (!b || !c || !slot) return fail(DSO_EINVAL, "null argument");
  dso_status st = check_ready(c);
  if (st != DSO_OK) return st;
  if (c->device != b->device || c->prec != b->prec)
    return fail(DSO_EINVAL, "the job's device and precision must be the batch's");
  for (const BatchSlot& s2 : b->slots)
    if (s2.live && s2.ctx == c) return fail(DSO_EINVAL, "the context is already in the batch");
  if (!std::isfinite(t) || !std::isfinite(dt) || dt == 0.0) return fail(DSO_EINVAL, "t and dt must be finite, dt != 0");
  const double ratio = t / dt, nr = std::round(ratio);
  if (nr < 0 || std::fabs(ratio - nr) > 1e-9 * std::fmax(1.0, std::fabs(ratio)))
    return fail(DSO_EINVAL, "t / dt must be a non-negative integer");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);  // the job's own work is done before the batch's stream takes over
  const int ol = c->max_line, ot = c->max_tile;
  c->max_line = kBatchMaxLine;
  c->max_tile = kBatchMaxTile;
  c->limits_tuned = true;  // the batch's limits, not tuned ones
  st = replan(c);
  if (st != DSO_OK) {
    c->max_line = ol;
    c->max_tile = ot;
    const dso_status back = replan(c);
    (void)back;
    return fail(DSO_EINVAL, "the job's grid is too large for a batch slot (lines of at most 1024 points, and "
                            "S x 2048 points on axis 0, after one split): propagate it alone");
  }
  BatchSlot s;
  try {
    st = ensure_coeffs(c);
    if (st == DSO_OK) st = ensure_tables(c, dt, false);
    if (st != DSO_OK) return st;
    for (int d = 0; d < c->Dv; ++d) {
      c->G[d][0] = batch_G(c, (int)c->nv[d], 1);
      c->G[d][1] = batch_G(c, (int)c->nv[d], c->S);
      c->variant[d][0] = c->variant[d][1] = 0;
    }
    c->tuned = true;  // the batch's tile layout, not the autotuner's
    c->plane_on = false;  // line passes only
    drop_graph(c);
    st = batch_list(c, step_passes(c, true), s.first);
    if (st == DSO_OK) st = batch_list(c, step_passes(c, false), s.mid);
    if (st == DSO_OK) st = batch_list(c, final_passes(c), s.fin);
    if (st != DSO_OK) return st;
  } catch (const std::exception& ex) {
    return fail(DSO_EINVAL, ex.what());
  }
  s.ctx = c;
  s.dt = dt;
  s.steps_total = (long long)nr;
  s.live = true;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i].live && !b->slots[i].ctx) {
      b->slots[i] = std::move(s);
      *slot = (int)i;
      return DSO_OK;
    }
  b->slots.push_back(std::move(s));
  *slot = (int)b->slots.size() - 1;
  return DSO_OK;
}

dso_status dso_batch_step(dso_batch* b, int* active) {
  NvtxRange nvtx("dso_batch_step");
  if (!b) return fail(DSO_EINVAL, "null batch");
  DeviceGuard g(b->device);
  // the work list: each unfinished job's passes for its next step (the
  // first-step list, or a middle step's; the final passes after its last)
  std::vector<BatchPass> passes;
  std::vector<std::pair<int, int>> span;  // per running slot: first pass index, count
  std::vector<int> running;
  for (size_t i = 0; i < b->slots.size(); ++i) {
    BatchSlot& s = b->slots[i];
    if (!s.live || s.steps_done >= s.steps_total) continue;
    const int start = (int)passes.size();
    const std::vector<BatchPass>& body = s.steps_done == 0 ? s.first : s.mid;
    passes.insert(passes.end(), body.begin(), body.end());
    if (s.steps_done + 1 == s.steps_total) passes.insert(passes.end(), s.fin.begin(), s.fin.end());
    span.emplace_back(start, (int)passes.size() - start);
    running.push_back((int)i);
  }
  int still = 0;
  if (!running.empty()) {
    // segments by round, then by job: a job's pass r - 1 precedes its pass r
    std::vector<BatchSeg> segs;
    std::vector<int> last_seg(span.size(), -1);
    int rounds = 0;
    for (auto& sp : span) rounds = std::max(rounds, sp.second);
    long long item = 0;
    size_t smem = 0;
    for (int r = 0; r < rounds; ++r)
      for (size_t j = 0; j < span.size(); ++j) {
        if (r >= span[j].second) continue;
        const int pi = span[j].first + r;
        const BatchPass& bp = passes[pi];
        BatchSeg sg;
        sg.item0 = item;
        sg.pass = pi;
        sg.prev = last_seg[j];
        last_seg[j] = (int)segs.size();
        segs.push_back(sg);
        item += bp.ntiles;
        const int Wi = 1 << std::min(bp.a.stride_log2, bp.a.G_log2);
        smem = std::max(smem, batch_tile_smem(bp.L, bp.SV, bp.a.G, Wi, b->prec == DSO_FP32));
      }
    CK(cudaStreamSynchronize(b->stream));  // the previous launch no longer reads the host copies
    b->h_pass.swap(passes);
    b->h_seg.swap(segs);
    dso_status st = batch_reserve(b, b->h_pass.size(), b->h_seg.size());
    if (st != DSO_OK) return st;
    CK(cudaMemcpyAsync(b->d_pass, b->h_pass.data(), b->h_pass.size() * sizeof(BatchPass), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemcpyAsync(b->d_seg, b->h_seg.data(), b->h_seg.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemsetAsync(b->d_done, 0, b->h_seg.size() * sizeof(unsigned), b->stream));
    CK(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), b->stream));
    CK(launch_batch_worklist(b->prec == DSO_FP32, b->d_seg, (int)b->h_seg.size(), b->d_pass, item, b->d_head,
                             b->d_done, b->d_err, smem, b->stream));
    b->launches += 1;
    for (int i : running) b->slots[i].steps_done += 1;
  }
  for (const BatchSlot& s : b->slots)
    if (s.live && s.steps_done < s.steps_total) ++still;
  if (active) *active = still;
  return DSO_OK;
}

dso_status dso_batch_sync(dso_batch* b) {
  if (!b) return fail(DSO_EINVAL, "null batch");
  DeviceGuard g(b->device);
  int h = 0;
  CK(cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  if (h != 0) {
    CK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
    return fail(DSO_ETIMEOUT, "a batch tile's bounded wait for its job's previous pass gave up (code " +
                                  std::to_string(h) + ")");
  }
  return DSO_OK;
}

dso_status dso_batch_slot_status(const dso_batch* b, int slot, int64_t* steps_done, int64_t* steps_total) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].live) return fail(DSO_EINVAL, "no such slot");
  if (steps_done) *steps_done = b->slots[slot].steps_done;
  if (steps_total) *steps_total = b->slots[slot].steps_total;
  return DSO_OK;
}

dso_status dso_batch_retire(dso_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].live) return fail(DSO_EINVAL, "no such slot");
  DeviceGuard g(b->device);
  CK(cudaStreamSynchronize(b->stream));  // the job's state is final before its context is handed back
  BatchSlot& s = b->slots[slot];
  s.ctx->tuned = false;  // used alone again, the context tunes its own tiles
  s.ctx->have_psi = true;
  s.live = false;
  s.ctx = nullptr;
  s.first.clear();
  s.mid.clear();
  s.fin.clear();
  return DSO_OK;
}

int64_t dso_batch_launch_count(const dso_batch* b) { return b ? b->launches : 0; }

int dso_batch_busy(const dso_batch* b) {
  if (!b) return fail(DSO_EINVAL, "null batch");
  DeviceGuard g(b->device);
  const cudaError_t e = cudaStreamQuery(b->stream);
  if (e == cudaSuccess) return 0;
  if (e == cudaErrorNotReady) return 1;
  return fail(DSO_ECUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
}

const char* dso_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace dso {

bool axis_pass_supported(int L, int SV) {
  if (L < 8 || L > DSO_MAX_LINE || (L & (L - 1))) return false;
  if (SV < 1 || SV > 4) return false;
  return (long long)SV * L <= 8192;
}

int axis_pass_max_tile_lines(int L, int SV) {
  const int maxt = (SV * L / 8 > 256) ? SV * L / 8 : 256;
  int g = (maxt * 8) / (SV * L);
  return g < 1 ? 1 : g;
}

bool axis_pass_tma_supported(int L, int SV, int G) {
  if (!axis_pass_supported(L, SV) || L > 256) return false;
  const int np = SV > 1 ? SV * (SV + 1) / 2 : 1;
  const long long smem = (long long)(SV + np) * G * L * 16 + (long long)L * 16 + 192;
  return SV * G * (L / 8) <= 256 && smem <= 220 * 1024 && encode_fn() != nullptr;
}

bool axis_pass_tmap_supported(int L, int SV, int G) {
  if (!axis_pass_supported(L, SV) || L > 256) return false;
  const int np = SV > 1 ? SV * (SV + 1) / 2 : 1;
  const long long smem = 2LL * (SV + np) * G * L * 16 + (long long)L * 16 + 192;
  return SV * G * (L / 8) <= 256 && smem <= 220 * 1024 && encode_fn() != nullptr;
}

bool axis_pass_reg_supported(int L, int SV, bool fp32, long long stride, bool dec0) {
  const int g = axis_pass_reg_lines(L, SV);
  if (g == 0 || (stride != 1 && stride < g)) return false;
  const int vpt = L == 128 ? 16 : 8, w = fp32 ? 2 : 4;
  // the amplitudes fit a thread's registers (reg_fits), all SV surfaces or,
  // with surface 0 decoupled, the block of the others (the split form)
  return SV * vpt * w <= 96 || (dec0 && SV >= 3 && (SV - 1) * vpt * w <= 96);
}

int axis_pass_reg_lines(int L, int SV) {
  if (SV < 1 || SV > DSO_MAX_SURFACES || (L != 32 && L != 64 && L != 128)) return 0;
  const int tpl = L == 32 ? RegPlan<32>::TPL : L == 64 ? RegPlan<64>::TPL : RegPlan<128>::TPL;
  return (SV == 1 ? reg_threads<1>() : reg_threads<2>()) / tpl;
}

bool axis_pass_pq_supported(int L, int SV, int G) {
  if (!axis_pass_supported(L, SV)) return false;
  const int np = SV > 1 ? SV * (SV + 1) / 2 : 1;
  const long long smem = (long long)(2 * SV + np) * G * L * 16;
  return SV * G * (L / 8) <= 256 && smem <= 200 * 1024;
}

cudaError_t launch_axis_pass(int L, int SV, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                             const TmaMaps* maps, cudaStream_t st) {
  switch (SV) {
    case 1: return launch_axis_pass_sv1(L, variant, a, ntiles, queue, maps, st);
    case 2: return launch_axis_pass_sv2(L, variant, a, ntiles, queue, maps, st);
    case 3: return launch_axis_pass_sv3(L, variant, a, ntiles, queue, maps, st);
    case 4: return launch_axis_pass_sv4(L, variant, a, ntiles, queue, maps, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dso
