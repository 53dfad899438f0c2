// Plan construction and the C ABI (include/fmm.h).
//
// The plan precomputes everything that depends only on the geometry (Sec. 2.2:
// the cell-centred scheme fixes the interaction displacements, so the
// Green's-function derivatives are tabulated once):
//  * the hierarchy extents (round-up halving, Sec. 2);
//  * Taylor coefficients of 1/|u + t| at every unit box offset u of the
//    interaction list, by the three-term recurrence
//        n |u|^2 b_g = -(2n-1) sum_i u_i b_{g-e_i} - (n-1) sum_i b_{g-2e_i},
//    n = |g| (derivatives of g = -1/r are then D_g = -g! b_g);
//  * the unit-box M2L operator Wt_u[beta][alpha] = (-1)^|alpha|
//    C(alpha+beta, alpha) (-b_{alpha+beta}(u)), laid out as column tiles of
//    the neighbour contraction (k_gemm_simt.cu);
//  * the near-field matrix g(x_t - x_s) per neighbour leaf box (eq. direct);
//  * the M2M / L2L shift pair lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fmm_internal.h"

using namespace fmmgb;

namespace {

thread_local std::string g_last_error;

fmm_status fail(fmm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CUDA_TRY(expr)                                                                           \
  do {                                                                                           \
    cudaError_t e__ = (expr);                                                                    \
    if (e__ != cudaSuccess) return fail(FMM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e__)); \
  } while (0)

struct MultiIndex {
  int p = 0, nc = 0;
  int mo = 0;  // multipole order limit (components above it take no part in M2L / M2P); p by default
  int lo = 0;  // local order limit of the M2L (p by default; mo of the forward in its transpose)
  std::vector<int> a, b, c;  // components, canonical order
  int index(int x, int y, int z) const {
    const int n = x + y + z;
    return n * (n + 1) * (n + 2) / 6 + (n - x) * (n - x + 1) / 2 + (n - x - y);
  }
  void init(int order) {
    p = mo = lo = order;
    a.clear(), b.clear(), c.clear();
    for (int n = 0; n <= p; ++n)
      for (int x = n; x >= 0; --x)
        for (int y = n - x; y >= 0; --y) {
          a.push_back(x), b.push_back(y), c.push_back(n - x - y);
        }
    nc = (int)a.size();
  }
};

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Taylor coefficients of 1/|u + t| in t for |g| <= p (canonical order).
void taylor_inv_r(const double u[3], const MultiIndex& mi, std::vector<double>& out) {
  out.assign(mi.nc, 0.0);
  const double r2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  out[0] = 1.0 / std::sqrt(r2);
  for (int k = 1; k < mi.nc; ++k) {
    const int g[3] = {mi.a[k], mi.b[k], mi.c[k]};
    const int n = g[0] + g[1] + g[2];
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
      int h[3] = {g[0], g[1], g[2]};
      if (g[i] >= 1) {
        h[i] = g[i] - 1;
        s -= (2.0 * n - 1.0) * u[i] * out[mi.index(h[0], h[1], h[2])];
      }
      if (g[i] >= 2) {
        h[i] = g[i] - 2;
        s -= (n - 1.0) * out[mi.index(h[0], h[1], h[2])];
      }
    }
    out[k] = s / (n * r2);
  }
}

int level_of_order(const MultiIndex& mi, int k) { return mi.a[k] + mi.b[k] + mi.c[k]; }

int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Harmonic (c <= 1) components in reduced order (order, then b + c, then c):
// the canonical index of each; their count up to order q is (q + 1)^2.
std::vector<int> harmonic_components(const MultiIndex& mi) {
  std::vector<int> r;
  for (int n = 0; n <= mi.p; ++n)
    for (int s = 0; s <= n; ++s)
      for (int c = 0; c <= 1 && c <= s; ++c) r.push_back(mi.index(n - s, s - c, c));
  return r;
}

enum Stage {
  ST_CHECK = 0,
  ST_P2M,
  ST_M2M,
  ST_L2L,
  ST_M2L,
  ST_NEAR,
  ST_LEAF,
  ST_FD,
  ST_ADJ_SRC,
  ST_SPLIT,
  ST_M2L_TC,
  ST_NEAR_TC,
  ST_COUNT
};
const char* kStageNames[ST_COUNT] = {"finite_check", "p2m",          "m2m",         "l2l",       "m2l", "near_field",
                                     "leaf_l2p",     "fd_accel",     "adjoint_source", "split_bf16", "m2l_tc", "near_field_tc"};
constexpr int kEventPool = 8192;

}  // namespace

struct fmm_plan_s {
  int dims[3] = {0, 0, 0};
  double dx = 1.0, G = 1.0;
  int p = 0, b = 0, nc = 0;
  fmm_opts opts{};
  int L = 0;
  int lmin = 0;  // first level with stored expansions
  Level lev[kMaxLevels];
  MultiIndex mi;

  // device memory
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t rho_box_off = 0, near_off = 0, work_off = 0;
  int* d_flag = nullptr;
  int8_t* d_mi = nullptr;
  int* d_m2m_start = nullptr;
  ShiftEntry* d_m2m = nullptr;
  int* d_l2l_start = nullptr;
  ShiftEntry* d_l2l = nullptr;
  // SIMT M2L weights (fp32 and/or fp64) and tile tables
  void* d_w_m2l_f32 = nullptr;
  void* d_w_m2l_f64 = nullptr;
  int* d_m2l_tile_k = nullptr;
  long long* d_m2l_tile_w = nullptr;
  int m2l_ntiles = 0;
  // near field
  void* d_w_near = nullptr;
  int* d_near_tile_k = nullptr;
  long long* d_near_tile_w = nullptr;
  int near_ntiles = 0;
  // tensor-core M2L and near field
  int tc_kind = -1;
  bool harm = false;  // harmonic compression of the tensor-core M2L/M2P (activation rows of nr components)
  bool harm_cc = false;  // harmonic compression of the CUDA-core M2L (Level::fold_off / lred_off)
  int nr = 0;         // (p + 1)^2
  int plane_nc() const { return harm ? nr : nc; }
  TcLaunch tc{};
  // mult_order < order: the M2L with the two limits swapped (multipoles to p,
  // locals to mult_order), which the adjoint solve runs (transposed = true)
  bool asym = false, transposed = false;
  void* d_w_m2l_f32_t = nullptr;
  void* d_w_m2l_f64_t = nullptr;
  int* d_m2l_tile_k_t = nullptr;
  long long* d_m2l_tile_w_t = nullptr;
  TcLaunch tc_t{};
  bool near_tc = false;
  std::vector<TcLaunch> tcn;  // near field: kTcMaxPasses passes per launch
  alignas(64) unsigned char map_near_hi[128];
  alignas(64) unsigned char map_near_lo[128];
  size_t rho_hi_off = 0, rho_lo_off = 0;
  size_t part_off = 0;  // neighbour-split partial sums of the small SIMT levels
  size_t part_cap = 0;  // bytes there
  // CUDA-core contraction variant of each M2L level and of the near field
  // (shape / neighbour split; fmm_plan_autotune times the candidates)
  struct SimtChoice {
    int shape = 0, dsplit = 1;
  };
  SimtChoice m2l_choice[kMaxLevels];
  SimtChoice near_choice;
  std::vector<int> h_m2l_tile_k, h_near_tile_k;
  alignas(64) unsigned char map_hi[kMaxLevels][128];
  alignas(64) unsigned char map_lo[kMaxLevels][128];
  // host-buffer staging for fmm_solve_host (set 0) and fmm_solve_host_many
  // (sets 0 and 1), its copy streams and events
  void* d_io_rho = nullptr;
  void* d_io_phi = nullptr;
  void* d_io_acc = nullptr;
  void* d_io_rho1 = nullptr;
  void* d_io_phi1 = nullptr;
  void* d_io_acc1 = nullptr;
  cudaStream_t io_in = nullptr, io_out = nullptr;
  cudaEvent_t io_ev[7] = {};  // [b] uploaded, [2 + b] solved, [4 + b] downloaded (set b), [6] start
  cudaStream_t last_stream = nullptr;
  // side stream of the concurrent far field (CUDA-core M2L levels), fork/join events
  cudaStream_t side = nullptr;
  int near_comps = 1;  // near-field columns per cell: potential, + 3 force components (analytic accel)
  // final-stage M2P (the paper's own final stage): leaf interaction list at the cell centres
  bool m2p = false, m2p_tc = false;
  size_t m2p_off = 0;  // [leaf parent][child][m2p_comps][b^3] potentials (scaled, x 1/b in the leaf kernel)
  int m2p_comps = 1;   // 4 with the analytic force: the potential and its three derivatives
  // transpose of the analytic force (fmm_solve_adjoint with grad_accel and
  // accel = 2): dipole P2M sources [3][cells] and the near field's transpose
  // over [w, -g/dx] x b^3 per box (CUDA cores), into one potential column
  size_t adj_dip_off = 0;
  void* d_w_near_adj = nullptr;
  int* d_near_adj_tile_k = nullptr;
  long long* d_near_adj_tile_w = nullptr;
  int near_adj_ntiles = 0;
  std::vector<int> h_near_adj_tile_k;
  const void* adj_g = nullptr;  // during an adjoint solve: the force's adjoint input [3][cells]
  void* d_w_m2p = nullptr;
  int* d_m2p_tile_k = nullptr;
  long long* d_m2p_tile_w = nullptr;
  int m2p_ntiles = 0;
  std::vector<int> h_m2p_tile_k;
  // transpose of the final-stage M2P (the adjoint solve): P2L from the
  // adjoint source's cells into the leaf locals, CUDA cores
  void* d_w_p2l = nullptr;
  int* d_p2l_tile_k = nullptr;
  long long* d_p2l_tile_w = nullptr;
  int p2l_ntiles = 0;
  std::vector<int> h_p2l_tile_k;
  TcLaunch tcm{};
  // prefix-schedule forms (k_nbr_tc.cu) of the M2L (and its transpose), the
  // final-stage M2P and the near field; the span forms above run where a
  // prefix schedule does not apply.  Where both exist, use_tp[] picks one
  // (TcSched: M2L, near field, M2P): defaults from measurement, then
  // fmm_plan_autotune times both.
  bool tp_m2l = false, tp_m2l_t = false, tp_m2p = false, tp_near = false;
  bool span_m2l = false, span_m2l_t = false, span_near = false, span_m2p = false;
  bool use_tp[3] = {true, false, true};
  // the dedicated near-field kernel of leaf 4 (k_near_tc.cu), used when
  // present unless another schedule is selected
  bool near4 = false, use_near4 = true;
  NearTcLaunch ntl{};
  bool inject_timeout = false;  // test hook (fmm_plan_debug_timeout): the next prefix launch starves its first stage
  TpLaunch tpl{}, tpl_t{}, tpm{}, tpn{};
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;

  bool f64_data() const { return opts.precision == FMM_FP64; }
  // SIMT M2L levels too small to fill the GPU run one CTA per neighbour.
  bool split_level(int l) const {
    const Level& lv = lev[l];
    const long long tiles = (long long)((lv.np[0] + 3) / 4) * ((lv.np[1] + 3) / 4) * ((lv.np[2] + 3) / 4);
    return !no_split && !lv.tc && tiles * m2l_ntiles < 2 * 152;
  }
  size_t esize() const { return f64_data() ? 8 : 4; }
  long long ncell() const { return (long long)dims[0] * dims[1] * dims[2]; }
  TreeTables tables() const {
    TreeTables t;
    t.mi = d_mi;
    t.m2m_start = d_m2m_start;
    t.m2m = d_m2m;
    t.l2l_start = d_l2l_start;
    t.l2l = d_l2l;
    t.p = p;
    t.nc = nc;
    t.b = b;
    return t;
  }
  void* M(int l) const { return arena + lev[l].m_off; }
  void* Lx(int l) const { return arena + lev[l].l_off; }

  // Device placement: cudaMalloc (plans) or a bump pointer inside a caller
  // supplied region (the allocation-free solve), where the tables can be
  // left as the previous call wrote them.
  unsigned char* static_base = nullptr;
  size_t static_cap = 0, static_used = 0;
  bool static_keep_tables = false;
  bool no_split = false;
  // Layout only (host checks of the batch tables): with static_base a
  // placeholder address and static_keep_tables set, plan_init then touches
  // no device memory.
  bool dry = false;

  fmm_status dev_alloc(size_t bytes, void** out) {
    if (static_base) {
      const size_t off = (static_used + 255) & ~(size_t)255;
      if (off + bytes > static_cap)
        return fail(FMM_ERR_ARG, "workspace of more than %zu bytes does not fit the %zu-byte static array",
                    off + bytes, static_cap);
      static_used = off + bytes;
      *out = static_base + off;
      return FMM_OK;
    }
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(FMM_ERR_ALLOC, "cudaMalloc(%zu) failed", bytes);
    }
    allocs.push_back(d);
    dev_bytes += bytes;
    *out = d;
    return FMM_OK;
  }

  template <typename T>
  fmm_status upload(const std::vector<T>& host, T** dptr, cudaStream_t s) {
    const size_t bytes = std::max<size_t>(host.size(), 1) * sizeof(T);
    void* d = nullptr;
    fmm_status st = dev_alloc(bytes, &d);
    if (st != FMM_OK) return st;
    if (!host.empty() && !static_keep_tables)
      CUDA_TRY(cudaMemcpyAsync(d, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    *dptr = static_cast<T*>(d);
    return FMM_OK;
  }
  void release() {
    cudaDeviceSynchronize();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    ev_fork = ev_join = nullptr;
    side = nullptr;
    for (void* d : allocs) cudaFree(d);
    allocs.clear();
    for (void* d : {d_io_rho, d_io_phi, d_io_acc, d_io_rho1, d_io_phi1, d_io_acc1})
      if (d) cudaFree(d);
    for (cudaEvent_t e : io_ev)
      if (e) cudaEventDestroy(e);
    if (io_in) cudaStreamDestroy(io_in);
    if (io_out) cudaStreamDestroy(io_out);
  }
};

namespace {

// Build the per-level extents (Sec. 2: halve with round-up to one box).
fmm_status build_levels(fmm_plan_t P) {
  int ext[kMaxLevels][3];
  int cnt = 1;
  for (int q = 0; q < 3; ++q) ext[0][q] = P->dims[q] / P->b;
  while (ext[cnt - 1][0] > 1 || ext[cnt - 1][1] > 1 || ext[cnt - 1][2] > 1) {
    if (cnt >= kMaxLevels) return fail(FMM_ERR_ARG, "grid too deep");
    for (int q = 0; q < 3; ++q) ext[cnt][q] = (ext[cnt - 1][q] + 1) / 2;
    ++cnt;
  }
  P->L = cnt - 1;
  for (int l = 0; l <= P->L; ++l) {
    Level& lv = P->lev[l];
    for (int q = 0; q < 3; ++q) {
      lv.n[q] = ext[P->L - l][q];
      lv.np[q] = (lv.n[q] + 1) / 2;
    }
    lv.nbox = (long long)lv.n[0] * lv.n[1] * lv.n[2];
    lv.npar = (long long)lv.np[0] * lv.np[1] * lv.np[2];
  }
  return FMM_OK;
}

// Taylor coefficients of 1/|u + t| at every unit offset u in [-3,3]^3 that
// the interaction list reaches (Chebyshev distance >= 2).
struct TaylorTable {
  std::vector<std::vector<double>> t = std::vector<std::vector<double>>(343);
  void build(const MultiIndex& mi) {
    for (int uz = -3; uz <= 3; ++uz)
      for (int uy = -3; uy <= 3; ++uy)
        for (int ux = -3; ux <= 3; ++ux) {
          const int cheb = std::max(std::abs(ux), std::max(std::abs(uy), std::abs(uz)));
          if (cheb < 2) continue;
          const double u[3] = {(double)ux, (double)uy, (double)uz};
          taylor_inv_r(u, mi, t[(uz + 3) * 49 + (uy + 3) * 7 + (ux + 3)]);
        }
  }
  const std::vector<double>& at(const int u[3]) const { return t[(u[2] + 3) * 49 + (u[1] + 3) * 7 + (u[0] + 3)]; }
};

// One entry of the unit-box M2L contraction: neighbour parent d (0..26),
// reduction index k = alpha*8 + source child, output n = beta*8 + target child.
//   W = (-1)^|alpha| C(alpha+beta, alpha) (-b_{alpha+beta}(u)),
//   u = c_target - c_source in child-box units = ct - cs - 2 d,
// zero outside the interaction list (Chebyshev(u) < 2) or past the
// truncation |alpha| + |beta| > p.
double m2l_entry(const MultiIndex& mi, const TaylorTable& tt, int d, int k, int n) {
  const int nc = mi.nc, p = mi.p;
  const int be = n / 8, ct = n % 8, al = k / 8, cs = k % 8;
  if (be >= nc || al >= nc) return 0.0;
  const int ob = level_of_order(mi, be), oa = level_of_order(mi, al);
  if (oa + ob > p || oa > mi.mo || ob > mi.lo) return 0.0;
  const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
  int u[3];
  for (int q = 0; q < 3; ++q) u[q] = ((ct >> q) & 1) - ((cs >> q) & 1) - 2 * D[q];
  const int cheb = std::max(std::abs(u[0]), std::max(std::abs(u[1]), std::abs(u[2])));
  if (cheb < 2) return 0.0;  // near neighbours are handled one level down
  const std::vector<double>& tb = tt.at(u);
  const int g = mi.index(mi.a[al] + mi.a[be], mi.b[al] + mi.b[be], mi.c[al] + mi.c[be]);
  const double mult = binom(mi.a[al] + mi.a[be], mi.a[al]) * binom(mi.b[al] + mi.b[be], mi.b[al]) *
                      binom(mi.c[al] + mi.c[be], mi.c[al]);
  return ((oa & 1) ? -1.0 : 1.0) * mult * (-tb[g]);
}

// Column tiles of the neighbour contraction for M2L on the CUDA cores:
// output column n = beta*8 + child; tile t covers beta in [4t, 4t+4) whose
// lowest order fixes the reduction prefix 8 * nc(p - order).  harm: rows
// and columns are the harmonic components ((q + 1)^2 up to order q: the
// folded multipoles in, the c <= 1 locals out).
template <typename T>
void m2l_weights(const MultiIndex& mi, const TaylorTable& tt, std::vector<T>& W, std::vector<int>& tile_k,
                 std::vector<long long>& tile_w, bool fill = true, bool harm = false) {
  const int p = mi.p;
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  auto count = [harm](int q) { return harm ? (q + 1) * (q + 1) : ncoef(q); };
  const int ncol = 8 * nk;
  const int ntiles = (ncol + kNTile - 1) / kNTile;
  tile_k.resize(ntiles);
  tile_w.resize(ntiles);
  long long off = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int beta0 = (t * kNTile) / 8;
    const int o = level_of_order(mi, harm ? red[beta0] : beta0);
    tile_k[t] = 8 * count(std::min(p - o, mi.mo));
    tile_w[t] = off;
    off += 27LL * tile_k[t] * kNTile;
  }
  W.assign((size_t)off, T(0));
  if (!fill) return;
  for (int t = 0; t < ntiles; ++t) {
    const int K = tile_k[t];
    for (int d = 0; d < 27; ++d) {
      T* blk = W.data() + tile_w[t] + (long long)d * K * kNTile;
      for (int k = 0; k < K; ++k)
        for (int j = 0; j < kNTile; ++j) {
          const int n = t * kNTile + j;
          if (!harm) {
            blk[(long long)k * kNTile + j] = (T)m2l_entry(mi, tt, d, k, n);
          } else if (n / 8 < nk && k / 8 < nk) {
            blk[(long long)k * kNTile + j] =
                (T)m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8);
          }
        }
    }
  }
}

uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_to_f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
float tf32_rn(double w) {
  float f = (float)w;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= ~0x1FFFu;
  std::memcpy(&f, &u, 4);
  return f;
}

// Tensor-core schedule: column groups (order blocks, orders 0 and 1 merged,
// split into <= 128-column pieces), passes of <= 512 TMEM columns, and for
// every (neighbour, 128-byte reduction chunk) the weight tiles of the groups
// whose prefix reaches that chunk.  Weight tiles are written in the exact
// shared-memory image the MMA reads: rows of 128 B, 16-byte chunks swizzled
// by (row mod 8), bf16 hi plane then lo plane (or one TF32 plane).
struct TcHost {
  std::vector<TcPass> pass;  // kTcMaxPasses per launch
  int npass = 0;
  int a_stages = 2;
  std::vector<unsigned char> W;
};

// A column group before packing: output columns [col0, col0 + ncols) that
// share one reduction prefix of length K.  Groups come in non-increasing K.
struct TcCols {
  int col0, ncols, K;
};

// Instruction descriptor of one MMA: M = 128, N = n, FP32 accumulators.
uint32_t host_idesc(int kind, int n) {
  const uint32_t ab = kind == TC_TF32 ? 2u : 1u;  // TF32 : BF16 operands, F32 accumulate, K-major, M = 128
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Packs passes, MMA spans and weight tiles for groups `gs`; `entry(d, k, n)`
// gives one weight of the contraction.  Tiles are written in the exact
// shared-memory image the MMA reads: rows of 128 B, 16-byte chunks swizzled by
// (row mod 8), bf16 hi plane then lo plane (or one TF32 plane).
//
// Issue balance: a tcgen05.mma costs tens of cycles to issue whatever its N,
// and narrow low-order groups with long reductions need the most of them.
// The accumulators of a pass are therefore shared out between kTcIssuers
// issuing threads (heaviest first, to the least-loaded issuer), and a group
// whose MMA steps exceed an even share is split along the reduction at a chunk
// boundary into two accumulators, which the epilogue adds in a fixed order.
// A bf16x3 pass with a single group (the near field) is split by product
// instead: hi*hi, hi*lo and lo*hi go to three issuers with their own
// accumulators and one weight plane each; where TMEM leaves room, the hi*hi
// reduction is also halved at a chunk boundary onto the fourth issuer.
//
// `long_sums`: one group per pass, so that every group is product-split, and
// one neighbour column (dx, dz) per accumulation segment.  The tensor cores
// add into their FP32 accumulators with truncation (round toward zero), which
// on a long same-signed sum (the near field of a large leaf box: 27 x b^3
// terms) leaves a bias of about half an ulp per MMA; short reductions per
// accumulator, summed by the epilogue with rounding to nearest, bound it.
// `max_passes`: passes the caller can launch (kTcMaxPasses per launch).
template <typename Entry>
bool build_tc_generic(int kind, const std::vector<TcCols>& gs, const Entry& entry, TcHost& H, int a_stages,
                      bool long_sums = false, int max_passes = kTcMaxPasses) {
  const int ring_budget = tc_ring_budget(kind, a_stages);
  H.a_stages = a_stages;
  const int chunk = kind == TC_BF16X3 ? 64 : 32;  // reduction values per 128-byte chunk
  const int kstep = chunk / 4;
  const int esz = kind == TC_BF16X3 ? 2 : 4;
  const int planes = kind == TC_BF16X3 ? 2 : 1;
  // MMA K steps of reduction range [k0, k1) (k0 chunk-aligned) in chunk j
  auto ksteps_in = [&](int k0, int k1, int j) {
    if (k1 <= j * chunk || k0 >= (j + 1) * chunk) return 0;
    return std::min(4, (k1 - j * chunk + kstep - 1) / kstep);
  };
  struct VGroup {
    int out;       // output group
    int k0, k1;    // reduction range
    int nm;        // TMEM columns
    int prod = 0;  // TcSpan::prod
    int q = 0;     // issuer
    int tmem = 0;
  };
  auto vsteps = [&](const VGroup& v) {
    int n = 0;
    for (int j = v.k0 / chunk; j * chunk < v.k1; ++j) n += ksteps_in(v.k0, v.k1, j);
    return n;
  };
  H.W.clear();
  H.pass.clear();
  H.npass = 0;
  size_t gi = 0;
  while (gi < gs.size()) {
    if (H.npass == max_passes) return false;
    H.pass.emplace_back();
    ++H.npass;
    TcPass& P = H.pass.back();
    std::memset(&P, 0, sizeof(P));
    P.seg_xz = long_sums ? 1 : 9;
    // output groups of this pass, in the given (non-increasing K) order, up to 512 TMEM columns
    int cols = 0;
    std::vector<VGroup> V;
    while (gi < gs.size() && P.ng < kTcMaxGroups && !(long_sums && P.ng == 1)) {
      const int nm = (gs[gi].ncols + 15) / 16 * 16;
      if (cols + nm > 512) break;
      if (P.ng > 0 && gs[gi].K > gs[gi - 1].K) return false;  // prefixes must shrink
      P.out_col0[P.ng] = gs[gi].col0;
      P.out_ncols[P.ng] = gs[gi].ncols;
      P.out_nmma[P.ng] = nm;
      P.out_tmem2[P.ng] = -1;
      P.out_tmem3[P.ng] = -1;
      P.out_tmem4[P.ng] = -1;
      V.push_back({P.ng, 0, gs[gi].K, nm});
      cols += nm;
      ++P.ng;
      ++gi;
    }
    if (P.ng == 0) return false;
    // a single bf16x3 group: one accumulator per product
    const bool prod_split = kind == TC_BF16X3 && V.size() == 1 && 3 * cols <= 512;
    // hi*hi and hi*lo share A_hi, and a tile's lo plane follows its hi plane:
    // one MMA of N = 2n over both planes computes them into adjacent
    // accumulators (an N = 64 MMA holds the tensor pipe about as long as an
    // N = 128 one, so this is two pipe slots a K step instead of three)
    const bool pair_hilo = prod_split && !long_sums && 2 * V[0].nm <= 256;
    if (pair_hilo) {
      VGroup v3 = V[0];
      v3.prod = 3;
      V[0].prod = 4;
      V[0].nm *= 2;
      V.push_back(v3);
      cols *= 3;
      P.out_tmem2[0] = P.out_tmem3[0] = 0;  // marked; placed below
    } else if (prod_split) {
      V[0].prod = 1;
      VGroup v2 = V[0], v3 = V[0];
      v2.prod = 2;
      v3.prod = 3;
      V.push_back(v2);
      V.push_back(v3);
      cols *= 3;
      P.out_tmem2[0] = P.out_tmem3[0] = 0;  // marked; placed below
      // hi*hi in two halves (chunk boundary nearest the middle of its steps)
      const int hs = vsteps(V[0]);
      int best = -1, bestd = 1 << 30;
      for (int kb = chunk; kb < V[0].k1; kb += chunk) {
        VGroup a = V[0];
        a.k1 = kb;
        const int d = std::abs(2 * vsteps(a) - hs);
        if (d < bestd) bestd = d, best = kb;
      }
      if (best > 0 && cols + V[0].nm <= 512) {
        VGroup v4 = V[0];
        v4.k0 = best;
        V[0].k1 = best;
        V.push_back(v4);
        cols += v4.nm;
        P.out_tmem4[0] = 0;  // marked; placed below
      }
    }
    // split the heaviest accumulators along the reduction while one exceeds an even share
    int total = 0;
    for (const VGroup& v : V) total += vsteps(v);
    const int share = (total + kTcIssuers - 1) / kTcIssuers;
    for (bool again = !prod_split; again;) {
      again = false;
      int h = -1;
      for (int i = 0; i < (int)V.size(); ++i)
        if (P.out_tmem2[V[i].out] == -1 && V[i].k0 == 0 && (h < 0 || vsteps(V[i]) > vsteps(V[h]))) h = i;
      if (h < 0 || vsteps(V[h]) <= share || cols + V[h].nm > 512) break;
      // chunk boundary that halves the steps best
      int best = -1, bestd = 1 << 30;
      const int hs = vsteps(V[h]);
      for (int kb = chunk; kb < V[h].k1; kb += chunk) {
        VGroup a = V[h];
        a.k1 = kb;
        const int d = std::abs(2 * vsteps(a) - hs);
        if (d < bestd) bestd = d, best = kb;
      }
      if (best < 0) break;
      VGroup b = V[h];
      b.k0 = best;
      V[h].k1 = best;
      P.out_tmem2[V[h].out] = 0;  // marked; placed below
      V.push_back(b);
      cols += b.nm;
      again = true;
    }
    // issuers: heaviest first, each to the least-loaded issuer
    {
      std::vector<int> order(V.size());
      for (size_t i = 0; i < V.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return vsteps(V[a]) > vsteps(V[b]); });
      int load[kTcIssuers] = {};
      for (int i : order) {
        int q = 0;
        for (int t = 1; t < kTcIssuers; ++t)
          if (load[t] < load[q]) q = t;
        V[i].q = q;
        load[q] += vsteps(V[i]);
      }
    }
    // TMEM layout: issuer by issuer; within an issuer, by reduction start, then K (adjacent
    // accumulators with the same start and K steps merge into one span)
    std::stable_sort(V.begin(), V.end(), [&](const VGroup& a, const VGroup& b) {
      if (a.q != b.q) return a.q < b.q;
      if (a.k0 != b.k0) return a.k0 < b.k0;
      return a.k1 > b.k1;
    });
    {
      int c = 0, kmax = 0;
      for (VGroup& v : V) {
        v.tmem = c;
        c += v.nm;
        kmax = std::max(kmax, v.k1);
        if (v.prod == 4) {  // hi*hi in the first half, hi*lo in the second
          P.out_tmem[v.out] = v.tmem;
          P.out_tmem2[v.out] = v.tmem + v.nm / 2;
        } else if (v.prod >= 2)
          (v.prod == 2 ? P.out_tmem2 : P.out_tmem3)[v.out] = v.tmem;
        else if (v.k0 == 0)
          P.out_tmem[v.out] = v.tmem;
        else
          (v.prod == 1 ? P.out_tmem4 : P.out_tmem2)[v.out] = v.tmem;
      }
      int alloc = 32;
      while (alloc < c) alloc *= 2;
      if (alloc > 512) return false;
      P.tmem_cols = alloc;
      P.nchunks = (kmax + chunk - 1) / chunk;
      if (P.nchunks > kTcMaxChunks) return false;
    }
    // spans per chunk and issuer, their tile offsets inside one neighbour block
    int ns = 0, off = 0;
    long long vol[kTcIssuers] = {};
    int biggest[kTcIssuers] = {};
    std::vector<std::vector<int>> span_v;  // accumulators of each span
    for (int j = 0; j < P.nchunks; ++j) {
      for (int q = 0; q < kTcIssuers; ++q) {
        P.span_idx[j][q] = ns;
        size_t i = 0;
        while (i < V.size()) {
          if (V[i].q != q || ksteps_in(V[i].k0, V[i].k1, j) == 0) {
            ++i;
            continue;
          }
          const int ks = ksteps_in(V[i].k0, V[i].k1, j);
          if (ns == kTcMaxSpans) return false;
          TcSpan& S = P.span[ns];
          S.tmem_col = V[i].tmem;
          S.n = 0;
          S.ksteps = ks;
          S.first = V[i].k0 / chunk;
          S.prod = V[i].prod;
          std::vector<int> members;
          const int k0 = V[i].k0;
          while (i < V.size() && V[i].q == q && V[i].k0 == k0 && V[i].prod == S.prod &&
                 ksteps_in(V[i].k0, V[i].k1, j) == ks && V[i].tmem == S.tmem_col + S.n &&
                 S.n + V[i].nm <= kTcMaxSpanN) {
            S.n += V[i].nm;
            members.push_back((int)i);
            ++i;
          }
          if (members.empty()) return false;
          S.w_off = off;
          S.idesc = host_idesc(kind, S.n);
          const int bytes = S.n * 128 * (S.prod ? 1 : planes);
          off += bytes;
          vol[q] += bytes;
          biggest[q] = std::max(biggest[q], bytes);
          span_v.push_back(members);
          ++ns;
        }
      }
      P.span_idx[j][kTcIssuers] = ns;
    }
    for (int q = 0; q <= kTcIssuers; ++q) P.span_idx[P.nchunks][q] = ns;
    // weight rings in proportion to the bytes each issuer streams, each able to hold its largest span
    {
      long long vt = 0;
      int need = 0;
      for (int q = 0; q < kTcIssuers; ++q) vt += vol[q], need += (biggest[q] + 1023) / 1024 * 1024;
      if (need > ring_budget) return false;
      int spare = ring_budget - need, given = 0;
      for (int q = 0; q < kTcIssuers; ++q) {
        const int base = (biggest[q] + 1023) / 1024 * 1024;
        const int extra = vt > 0 ? (int)((double)spare * (double)vol[q] / (double)vt) / 1024 * 1024 : 0;
        P.ring_bytes[q] = vol[q] > 0 ? base + extra : 0;
        given += P.ring_bytes[q];
      }
      for (int q = 0; q < kTcIssuers && given < ring_budget; ++q)  // leftover to the busiest ring
        if (vol[q] > 0 && vol[q] == *std::max_element(vol, vol + kTcIssuers)) {
          P.ring_bytes[q] += (ring_budget - given) / 1024 * 1024;
          break;
        }
    }
    P.bytes_per_d = off;
    P.w_base = (long long)H.W.size();
    H.W.resize(H.W.size() + (size_t)27 * P.bytes_per_d, 0);
    for (int d = 0; d < 27; ++d)
      for (int j = 0; j < P.nchunks; ++j)
        for (int si = P.span_idx[j][0]; si < P.span_idx[j][kTcIssuers]; ++si) {
          const TcSpan& S = P.span[si];
          unsigned char* tile = H.W.data() + P.w_base + (size_t)d * P.bytes_per_d + S.w_off;
          int row0 = 0;
          for (int vi : span_v[si]) {
            const VGroup& v = V[vi];
            for (int r = 0; r < P.out_ncols[v.out]; ++r) {
              const int n = P.out_col0[v.out] + r, row = row0 + r;
              for (int e = 0; e < S.ksteps * kstep; ++e) {
                const int k = j * chunk + e;
                if (k < v.k0 || k >= v.k1) continue;
                const double w = entry(d, k, n);
                if (w == 0.0) continue;
                const int byte = e * esz;
                const size_t o = (size_t)row * 128 + (size_t)((((byte >> 4) ^ (row & 7)) << 4) | (byte & 15));
                if (kind == TC_BF16X3) {
                  const uint16_t h = bf16_rn((float)w);
                  const uint16_t l = bf16_rn((float)(w - (double)bf16_to_f(h)));
                  if (S.prod == 0) {
                    std::memcpy(tile + o, &h, 2);
                    std::memcpy(tile + (size_t)S.n * 128 + o, &l, 2);
                  } else if (S.prod == 4) {  // hi rows, then the lo rows (half a multiple of 8: same swizzle)
                    std::memcpy(tile + o, &h, 2);
                    std::memcpy(tile + (size_t)(v.nm / 2) * 128 + o, &l, 2);
                  } else {  // the one plane this product multiplies
                    std::memcpy(tile + o, S.prod == 2 ? &l : &h, 2);
                  }
                } else {
                  const float t = tf32_rn(w);
                  std::memcpy(tile + o, &t, 4);
                }
              }
            }
            row0 += v.nm;
          }
        }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Prefix schedule of the tensor-core contraction (k_nbr_tc.cu).
//
// Output column n (0 <= n < kcol.size()) reduces over k < kcol[n], with kcol
// non-increasing, so K step s (kstep reduction values) is needed by the
// column prefix of those with kcol[n] > s * kstep.  The columns are split
// into passes (contiguous ranges, at most 512 TMEM columns each) by a cost
// model of the tensor pipe measured on GB300: an MMA of M = 128, K = 16 costs
// max(40, 32 + N / 4, N / 2) cycles.  Within a pass, K step s is one MMA per
// product over its prefix (N <= 256 per instruction), into
//   D  for s < l2_step (hi*hi, hi*lo, lo*hi; or, "fused" when the prefix is
//      narrow: hi*hi and hi*lo as one MMA over [lo rows reversed; hi rows]
//      into E and D, then lo*hi into D),
//   L2 for s >= l2_step,
// so that the FP32 accumulators of the lowest columns (the longest sums)
// each take about half the MMAs: the tensor cores add with truncation.
// The weight blocks of a K step (32-byte rows, 32-byte swizzle) are packed
// in MMA order into pieces of at most kTpPieceBytes that never cross a
// 128-byte activation chunk; the program of MMAs is the same for every
// (dx, dz) neighbour column, only the weights differ.
struct TpHost {
  std::vector<TpPass> pass;
  int a_stages = 2, w_slots = 0;
  int owner_slot0[kTpIssuers] = {}, owner_nslots[kTpIssuers] = {};
  std::vector<unsigned char> W;
};

// Tensor-pipe cycles of one MMA (M = 128, K = 16 bf16 / 8 TF32) of N columns.
double tp_mma_cycles(int n) { return std::max(40.0, std::max(32.0 + n / 4.0, n / 2.0)); }

// MMA shapes (first accumulator column, N) the schedule issues: N <= 128 at
// any 16-column boundary, or N a multiple of 32 up to 256 filling from column
// 0 or 256 without crossing the next 256-column boundary.  (Wider MMAs at
// other columns faulted on GB300; these are the forms that have run.)
bool tp_shape_ok(int tcol, int n) {
  if (n < 16 || n % 16 || tcol < 0 || tcol % 16) return false;
  if (n <= 128) return true;
  return n % 32 == 0 && n <= 256 && (tcol == 0 || tcol == 256);
}

struct TpStepPlan {
  int n = 0;         // prefix columns (multiple of 16)
  int region = 0;    // 0 D, 1 fused (E + D), 2 L2, 3 fused with lo*hi into L2
};

struct TpPassPlan {
  int c0 = 0, c1 = 0;   // output columns
  int S = 0;            // K steps
  int D = 0, E = 0, W2 = 0, l2_step = 0;
  int chain = 0;        // MMAs into the busiest accumulator column per tile
  double cycles = 0;    // per tile
  std::vector<TpStepPlan> steps;
};

// Plans one pass over columns [c0, c1); false if it does not fit.
bool tp_plan_pass(int kind, const std::vector<int>& kcol, int c0, int c1, TpPassPlan& out) {
  const bool split = kind == TC_BF16X3;
  const int kstep = split ? 16 : 8, products = split ? 3 : 1;
  TpPassPlan P;
  P.c0 = c0, P.c1 = c1;
  P.D = (c1 - c0 + 15) / 16 * 16;
  if (P.D > 512 || c1 <= c0) return false;
  P.S = (kcol[c0] + kstep - 1) / kstep;
  if (P.S <= 0) return false;
  std::vector<int> N(P.S);
  for (int s = 0; s < P.S; ++s) {
    int n = 0;
    while (c0 + n < c1 && kcol[c0 + n] > s * kstep) ++n;
    N[s] = (n + 15) / 16 * 16;
  }
  auto unfused = [&](int n) {
    double c = 0;
    for (int o = 0; o < n; o += 128) c += tp_mma_cycles(std::min(128, n - o));
    return products * c;
  };
  const double fused_gain_min = 1.0;
  // a fused step of N columns issues 2N from column E - N (E: the E region)
  auto fusable = [](int n, int E) { return n <= E && tp_shape_ok(E - n, 2 * n); };
  // candidates: l2_step from S (no L2) down; E from the fusable steps that fit
  TpPassPlan best;
  bool have = false;
  for (int s2 = P.S; s2 >= 1; --s2) {
    const int W2 = s2 < P.S ? N[s2] : 0;
    if (P.D + W2 > 512) continue;
    const int ebudget = std::min(128, 512 - P.D - W2);
    // E: the widest fusable prefix that pays (each candidate width checked
    // against the shapes of every step fused under it)
    int E = 0;
    double best_gain = 0;
    if (split)
      for (int cand = 16; cand <= ebudget; cand += 16) {
        double gain = 0;
        for (int s = 0; s < s2; ++s)
          if (fusable(N[s], cand))
            gain += std::max(0.0, unfused(N[s]) - (tp_mma_cycles(2 * N[s]) + tp_mma_cycles(N[s])));
        if (gain > best_gain + fused_gain_min) best_gain = gain, E = cand;
      }
    TpPassPlan c = P;
    c.W2 = W2, c.E = E, c.l2_step = s2;
    c.steps.assign(P.S, {});
    int chainD = 0, chainL = 0;
    double cyc = 0;
    for (int s = 0; s < P.S; ++s) {
      TpStepPlan& st = c.steps[s];
      st.n = N[s];
      if (s >= s2) {
        st.region = 2;
        chainL += products;
        cyc += unfused(N[s]);
      } else if (E > 0 && fusable(N[s], E) &&
                 tp_mma_cycles(2 * N[s]) + tp_mma_cycles(N[s]) + fused_gain_min < unfused(N[s])) {
        st.region = 1;
        chainD += 2;
        cyc += tp_mma_cycles(2 * N[s]) + tp_mma_cycles(N[s]);
      } else {
        st.region = 0;
        if (N[s] > 0) chainD += products;
        cyc += unfused(N[s]);
      }
    }
    c.chain = 27 * std::max(chainD, chainL);
    c.cycles = 27 * cyc;
    // prefer chains within ~1100 MMAs (the accuracy of the span schedule's
    // split accumulators), then the fewest cycles
    auto score = [](const TpPassPlan& x) { return x.cycles * (x.chain > 1100 ? 1.0 + (x.chain - 1100) / 1100.0 : 1.0); };
    if (!have || score(c) < score(best)) best = c, have = true;
  }
  if (!have) return false;
  // with no late-step region, a fused step's lo*hi gets the L2 region to
  // itself when the columns fit: the D accumulators then take hi*hi alone
  if (best.l2_step == best.S && best.E > 0 && best.E + best.D + best.E <= 512) {
    best.W2 = best.E;
    int chainD = 0, chainL = 0;
    for (TpStepPlan& st : best.steps) {
      if (st.region == 1) st.region = 3, ++chainL;
      chainD += st.region == 0 ? products : 1;
    }
    best.chain = 27 * std::max(chainD, chainL);
  }
  out = best;
  return true;
}

// Builds passes, MMA programs and packed weights; entry(d, k, n) is the
// weight of the contraction (0 beyond kcol[n] and past the row length klen).
template <typename Entry>
bool build_tp_generic(int kind, const std::vector<int>& kcol, int klen, const Entry& entry, TpHost& H,
                      int max_chain = 2100) {
  const bool split = kind == TC_BF16X3;
  const int kstep = split ? 16 : 8, esz = split ? 2 : 4;
  const int ncols = (int)kcol.size();
  if (ncols == 0) return false;
  for (int n = 1; n < ncols; ++n)
    if (kcol[n] > kcol[n - 1]) return false;  // prefixes must shrink
  // candidate pass boundaries: where the reduction length changes (multiples of 8)
  std::vector<int> bnd{0};
  for (int n = 1; n < ncols; ++n)
    if (kcol[n] != kcol[n - 1] && n % 8 == 0) bnd.push_back(n);
  bnd.push_back(ncols);
  const int nb = (int)bnd.size();
  // copy costs per tile (cycles): activation boxes at ~50 B/clk, weights at ~70 B/clk
  const int planes = split ? 2 : 1;
  auto pass_cost = [&](const TpPassPlan& pp) {
    const int nch = (pp.S + 3) / 4;
    const double a_bytes = 9.0 * nch * planes * kTcAPlaneBytes;
    double w_bytes = 0;
    for (const TpStepPlan& st : pp.steps) w_bytes += 27.0 * st.n * 32 * planes;
    return std::max(pp.cycles, a_bytes / 50.0 + w_bytes / 70.0) + 4000.0;  // + epilogue and pipeline fill
  };
  // dp over boundaries: best[i][np] = cost of columns [0, bnd[i]) in np passes
  const double inf = 1e300;
  std::vector<std::vector<double>> best(nb, std::vector<double>(kTpMaxPasses + 1, inf));
  std::vector<std::vector<int>> from(nb, std::vector<int>(kTpMaxPasses + 1, -1));
  std::vector<std::vector<TpPassPlan>> plan_of(nb, std::vector<TpPassPlan>(nb));
  std::vector<std::vector<char>> ok_of(nb, std::vector<char>(nb, 0));
  for (int i = 0; i < nb; ++i)
    for (int j = i + 1; j < nb; ++j)
      if (tp_plan_pass(kind, kcol, bnd[i], bnd[j], plan_of[i][j]) && plan_of[i][j].chain <= max_chain) ok_of[i][j] = 1;
  best[0][0] = 0;
  for (int j = 1; j < nb; ++j)
    for (int np = 1; np <= kTpMaxPasses; ++np)
      for (int i = 0; i < j; ++i)
        if (ok_of[i][j] && best[i][np - 1] < inf) {
          const double c = best[i][np - 1] + pass_cost(plan_of[i][j]);
          if (c < best[j][np]) best[j][np] = c, from[j][np] = i;
        }
  int npass = -1;
  for (int np = 1; np <= kTpMaxPasses; ++np)
    if (best[nb - 1][np] < inf && (npass < 0 || best[nb - 1][np] < best[nb - 1][npass])) npass = np;
  if (npass < 0) return false;
  std::vector<TpPassPlan> plans(npass);
  for (int j = nb - 1, np = npass; np > 0; --np) {
    const int i = from[j][np];
    plans[np - 1] = plan_of[i][j];
    j = i;
  }
  H.pass.assign(npass, TpPass{});
  H.W.clear();
  H.a_stages = split ? 2 : 3;
  H.w_slots = tp_w_slots(kind, H.a_stages);
  if (H.w_slots < kTpIssuers) return false;
  for (int ps = 0; ps < npass; ++ps) {
    const TpPassPlan& pp = plans[ps];
    TpPass& T = H.pass[ps];
    std::memset(&T, 0, sizeof(T));
    T.col0 = pp.c0;
    T.ncols = pp.c1 - pp.c0;
    T.nchunks = (pp.S + 3) / 4;
    if (T.nchunks > kTpMaxChunks) return false;
    T.tmem_cols = (pp.E + pp.D + pp.W2 + 15) / 16 * 16;
    T.nbuf = 2 * T.tmem_cols <= 512 ? 2 : 1;
    T.ngroups = (T.ncols + 15) / 16;
    if (T.ngroups > kTpMaxGroups) return false;
    for (int g = 0; g < T.ngroups; ++g) {
      T.grp_d[g] = (int16_t)(pp.E + 16 * g);
      T.grp_e[g] = (int16_t)(16 * g + 16 <= pp.E ? pp.E - 16 - 16 * g : -1);
      T.grp_l2[g] = (int16_t)(16 * g + 16 <= pp.W2 ? pp.E + pp.D + 16 * g : -1);
    }
    // Units: the MMAs reading one weight block of one K step.  A unit's
    // accumulator columns lie in one ownership group: the first 128 columns
    // of D together with E (and L2 when it holds the fused steps' lo*hi), a
    // later 128-column chunk of D, or L2 when it holds the late K steps.
    struct Unit {
      int s, dy, form, tcol, n, tcol2;
      int group;
      std::vector<int> row_col;    // output column (pass-relative) of each block row
      std::vector<int> row_plane;  // 0 hi, 1 lo
    };
    const bool l2_late = pp.l2_step < pp.S;  // L2 holds late K steps (else: the fused lo*hi, or nothing)
    const int ngroups_d = (pp.D + 127) / 128;
    const int g_l2 = l2_late ? ngroups_d : -1;
    const int ngrp = ngroups_d + (l2_late ? 1 : 0);
    auto step_units = [&](int s, int dy) {
      std::vector<Unit> out;
      const TpStepPlan& st = pp.steps[s];
      const int n = st.n;
      if (st.region == 1 || st.region == 3) {  // fused: [lo rows reversed; hi rows]
        Unit u{s, dy, 1, pp.E - n, n, st.region == 3 ? pp.E + pp.D : pp.E, 0, {}, {}};
        for (int r = 0; r < n; ++r) u.row_col.push_back(n - 1 - r), u.row_plane.push_back(1);
        for (int r = 0; r < n; ++r) u.row_col.push_back(r), u.row_plane.push_back(0);
        out.push_back(u);
        return out;
      }
      const int base = st.region == 2 ? pp.E + pp.D : pp.E;
      for (int o = 0; o < n; o += 128) {
        const int m = std::min(128, n - o);
        Unit u{s, dy, split ? 0 : 2, base + o, m, 0, st.region == 2 ? g_l2 : o / 128, {}, {}};
        for (int pl = 0; pl < (split ? 2 : 1); ++pl)
          for (int r = 0; r < m; ++r) u.row_col.push_back(o + r), u.row_plane.push_back(pl);
        out.push_back(u);
      }
      return out;
    };
    // ownership groups -> issuers: heaviest first, each to the least-loaded issuer
    std::vector<long long> gload(ngrp, 0);
    for (int s = 0; s < pp.S; ++s)
      for (const Unit& u : step_units(s, 0)) gload[u.group] += u.form == 0 ? 3 : u.form == 1 ? 2 : 1;
    std::vector<int> owner(ngrp, 0);
    {
      std::vector<int> order(ngrp);
      for (int g = 0; g < ngrp; ++g) order[g] = g;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gload[a] > gload[b]; });
      long long load[kTpIssuers] = {};
      for (int g : order) {
        int q = 0;
        for (int t = 1; t < kTpIssuers; ++t)
          if (load[t] < load[q]) q = t;
        owner[g] = q;
        load[q] += gload[g];
      }
    }
    // pieces: per chunk, each owner's units packed in (dy, K step) order; a
    // piece holds one owner's blocks; the pieces of a chunk are then ordered
    // by their first unit's (dy, K step), so the ring fills in the order the
    // owners read
    struct Piece {
      int owner, key, len;
      std::vector<Unit> units;
      std::vector<int> offs;
    };
    std::vector<Piece> pieces;
    std::vector<uint32_t> prog;
    std::vector<int> piece_unit{0};
    for (int j = 0; j < T.nchunks; ++j) {
      T.chunk_piece[j] = (int16_t)pieces.size();
      std::vector<Piece> cp;
      std::vector<int> open(kTpIssuers, -1);
      for (int dy = 0; dy < 3; ++dy)
        for (int s = 4 * j; s < std::min(pp.S, 4 * j + 4); ++s)
          for (Unit& u : step_units(s, dy)) {
            const int q = owner[u.group];
            const int bytes = (int)u.row_col.size() * 32;
            if (bytes > kTpPieceBytes) return false;
            int& o = open[q];
            if (o < 0 || cp[o].len + bytes > kTpPieceBytes) {
              cp.push_back(Piece{q, dy * 4 + (s - 4 * j), 0, {}, {}});
              o = (int)cp.size() - 1;
            }
            cp[o].offs.push_back(cp[o].len);
            cp[o].len += bytes;
            cp[o].units.push_back(u);
          }
      std::stable_sort(cp.begin(), cp.end(), [](const Piece& a, const Piece& b) { return a.key < b.key; });
      for (Piece& pc : cp) pieces.push_back(std::move(pc));
    }
    T.chunk_piece[T.nchunks] = (int16_t)pieces.size();
    T.npieces = (int)pieces.size();
    if (T.npieces > kTpMaxPieces) return false;
    for (int k = 0; k < T.npieces; ++k) {
      const Piece& pc = pieces[k];
      T.piece_len16[k] = (uint16_t)(pc.len / 16);
      T.piece_owner[k] = (int8_t)pc.owner;
      T.piece_unit[k] = (int16_t)prog.size();
      for (size_t i = 0; i < pc.units.size(); ++i) {
        const Unit& u = pc.units[i];
        const int nn = u.form == 1 ? 2 * u.n : u.n;
        if (!tp_shape_ok(u.tcol, nn) || u.tcol + nn > T.tmem_cols) return false;
        if (u.form == 1 && (!tp_shape_ok(u.tcol2, u.n) || u.tcol2 + u.n > T.tmem_cols)) return false;
        prog.push_back(tp_unit(pc.offs[i], u.s % 4, u.dy, u.form, u.tcol, u.n, u.tcol2));
      }
    }
    T.piece_unit[T.npieces] = (int16_t)prog.size();
    if ((int)prog.size() > kTpMaxUnits) return false;
    for (size_t m = 0; m < prog.size(); ++m) T.unit[m] = prog[m];
    // weights: [dx, dz column][piece] x kTpPieceBytes, in the 32-byte-row,
    // 32-byte-swizzle image the MMAs read
    T.w_base = (long long)H.W.size();
    H.W.resize(H.W.size() + (size_t)9 * T.npieces * kTpPieceBytes, 0);
    for (int xz = 0; xz < 9; ++xz) {
      const int dx = xz % 3 - 1, dz = xz / 3 - 1;
      for (int k = 0; k < T.npieces; ++k) {
        const Piece& pc = pieces[k];
        for (size_t i = 0; i < pc.units.size(); ++i) {
          const Unit& u = pc.units[i];
          const int d = (dx + 1) + 3 * u.dy + 9 * (dz + 1);
          unsigned char* blk =
              H.W.data() + T.w_base + ((size_t)xz * T.npieces + k) * kTpPieceBytes + pc.offs[i];
          for (int r = 0; r < (int)u.row_col.size(); ++r) {
            const int nrel = u.row_col[r], n = pp.c0 + nrel;
            if (nrel < 0 || n >= pp.c1) continue;
            for (int e = 0; e < kstep; ++e) {
              const int kk = u.s * kstep + e;
              if (kk >= kcol[n] || kk >= klen) continue;
              const double w = entry(d, kk, n);
              if (w == 0.0) continue;
              const int byte = e * esz;
              const size_t o = (size_t)r * 32 + (size_t)((((byte >> 4) ^ ((r >> 2) & 1)) << 4) | (byte & 15));
              if (split) {
                const uint16_t h = bf16_rn((float)w);
                const uint16_t l = bf16_rn((float)(w - (double)bf16_to_f(h)));
                std::memcpy(blk + o, u.row_plane[r] ? &l : &h, 2);
              } else {
                const float t = tf32_rn(w);
                std::memcpy(blk + o, &t, 4);
              }
            }
          }
        }
      }
    }
  }
  // owner rings: every owner with pieces gets a slot, the rest go to the
  // owners in proportion to the bytes they stream (largest remainder)
  {
    double bytes[kTpIssuers] = {};
    for (const TpPass& T : H.pass)
      for (int k = 0; k < T.npieces; ++k) bytes[T.piece_owner[k]] += T.piece_len16[k] * 16.0;
    int ns[kTpIssuers] = {}, used = 0;
    double tot = 0;
    for (int q = 0; q < kTpIssuers; ++q) {
      tot += bytes[q];
      if (bytes[q] > 0) ns[q] = 1, ++used;
    }
    if (used > H.w_slots) return false;
    while (used < H.w_slots) {
      int best = -1;
      double bd = -1;
      for (int q = 0; q < kTpIssuers; ++q)
        if (bytes[q] > 0) {
          const double deficit = bytes[q] / tot * H.w_slots - ns[q];
          if (deficit > bd) bd = deficit, best = q;
        }
      ++ns[best];
      ++used;
    }
    int s0 = 0;
    for (int q = 0; q < kTpIssuers; ++q) {
      H.owner_slot0[q] = s0;
      H.owner_nslots[q] = ns[q];
      s0 += ns[q];
    }
  }
  // one accumulator-set layout for every pass of the launch: a CTA moving
  // from one pass to the next reuses the sets in the same places, so the
  // acc_empty barriers of a set cover its whole column range
  int tmax = 0;
  for (const TpPass& T : H.pass) tmax = std::max(tmax, T.tmem_cols);
  for (TpPass& T : H.pass) {
    T.tmem_cols = tmax;
    T.nbuf = 2 * tmax <= 512 ? 2 : 1;
  }
  return true;
}

// M2L groups: order blocks (orders 0 and 1 merged), each with the prefix
// 8 nc(p - lowest order), split into pieces of <= 128 columns.  harm: rows
// and columns are the harmonic components only ((q + 1)^2 up to order q; the
// multipoles arrive folded and the epilogue's column map places the locals).
bool build_tc(const MultiIndex& mi, const TaylorTable& tt, int kind, TcHost& H, bool harm) {
  const int p = mi.p;
  auto count = [harm](int q) { return harm ? (q + 1) * (q + 1) : ncoef(q); };
  std::vector<TcCols> gs;
  for (int m = 0; m <= p;) {
    const int o_hi = (m == 0 && p >= 1) ? 1 : m;
    const int col0 = m == 0 ? 0 : 8 * count(m - 1), col1 = 8 * count(o_hi);
    const int K = 8 * count(std::min(p - m, mi.mo));
    const int total = col1 - col0;
    const int pieces = (total + kTcMaxGroupN - 1) / kTcMaxGroupN;
    const int per = ((total + pieces - 1) / pieces + 15) / 16 * 16;
    for (int c = col0; c < col1; c += per) gs.push_back({c, std::min(per, col1 - c), K});
    m = o_hi + 1;
  }
  // Two activation stages (the boxes have a producer thread of their own);
  // the weight rings take the rest of shared memory: the kernel is bound by
  // the number of weight tiles in flight against the L2 round trip.
  const std::vector<int> red = harmonic_components(mi);
  auto entry = [&](int d, int k, int n) {
    if (!harm) return m2l_entry(mi, tt, d, k, n);
    if (k / 8 >= (int)red.size() || n / 8 >= (int)red.size()) return 0.0;
    return m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8);
  };
  return build_tc_generic(kind, gs, entry, H, 2);
}

// One near-field weight (eq. direct, cell units) between source cell s of the
// neighbour leaf box at offset D and output column n = q * b^3 + t (target
// cell t): q = 0 the potential kernel g(r) (-1 for the cell itself); q = 1..3
// the force kernel d/dx_q g(r) = r_q / |r|^3 (0 for the cell itself), with
// r = x_t - x_s.
double near_entry(int b, const int D[3], int s, int n) {
  const int b3 = b * b * b;
  const int q = n / b3, t = n % b3;
  const int tp[3] = {t % b, (t / b) % b, t / (b * b)};
  const int sp[3] = {s % b, (s / b) % b, s / (b * b)};
  double r[3], r2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    r[a] = (double)(tp[a] - sp[a] - b * D[a]);
    r2 += r[a] * r[a];
  }
  if (q == 0) return r2 == 0.0 ? -1.0 : -1.0 / std::sqrt(r2);
  return r2 == 0.0 ? 0.0 : r[q - 1] / (r2 * std::sqrt(r2));
}

// Weights of the dedicated leaf-4 near-field kernel (k_near_tc.cu): per
// neighbour d the B operand's shared-memory image of W_d[k][n] =
// near_entry(d, k, n): row n (target cell) of 128 B holds the 64 source
// cells k, 16-byte chunks swizzled by (n mod 8); the bf16 hi plane, then the
// lo plane (w - hi rounded to bf16).
void near4_weights(std::vector<unsigned char>& W4) {
  W4.assign((size_t)27 * kNtPieceBytes, 0);
  for (int d = 0; d < 27; ++d) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    unsigned char* piece = W4.data() + (size_t)d * kNtPieceBytes;
    for (int n = 0; n < 64; ++n)
      for (int k = 0; k < 64; ++k) {
        const double w = near_entry(4, D, k, n);
        const uint16_t h = bf16_rn((float)w);
        const uint16_t l = bf16_rn((float)(w - (double)bf16_to_f(h)));
        const int byte = 2 * k;
        const size_t o = (size_t)n * 128 + (size_t)((((byte >> 4) ^ (n & 7)) << 4) | (byte & 15));
        std::memcpy(piece + o, &h, 2);
        std::memcpy(piece + kNtPieceBytes / 2 + o, &l, 2);
      }
  }
}

// Near field (eq. direct) as the same contraction over leaf boxes: column n =
// (component, target cell), reduction k = source cell of neighbour box d,
// weight near_entry(d, k, n).
bool build_tc_near(int b, int comps, int kind, TcHost& H) {
  const int b3 = b * b * b;
  std::vector<TcCols> gs;
  // groups of up to 128 columns: an MMA narrower than 64 columns holds the
  // tensor pipe as long as a 64-column one, so each b = 4 component is one group
  const int per = std::min(kTcMaxGroupN, b3);
  for (int c = 0; c < comps * b3; c += per) gs.push_back({c, std::min(per, comps * b3 - c), b3});
  auto entry = [b](int d, int k, int n) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    return near_entry(b, D, k, n);
  };
  // b >= 8: 27 x 512 same-signed terms per potential, too long a sum for one
  // truncating accumulator (bias ~3e-5); one product-split group per pass,
  // drained after every neighbour column, over as many launches as it takes
  const bool long_sums = b3 > 64;
  return build_tc_generic(kind, gs, entry, H, 2, long_sums, long_sums ? kTcMaxNearLaunches * kTcMaxPasses : kTcMaxPasses);
}

// Final-stage M2P (Sec. 4) as the same neighbour contraction over the leaf
// parents: reduction k = alpha*8 + source child (the parent-blocked multipole
// row), output n = target child * b^3 + cell, weight
//   W = (-1)^|alpha| (-b_alpha(u + e)),
// u = c_target - c_source in leaf-box units (ct - cs - 2d, interaction list
// only: Chebyshev(u) >= 2), e = the cell centre in the target box (box
// units), b_alpha the Taylor coefficients of 1/|r|; the result, times 1/h,
// is the cell potential of the source box's scaled multipoles.
struct M2pTable {
  int b = 0;
  std::vector<std::vector<double>> t;  // [u (7^3)][cell] -> nc coefficients
  void build(const MultiIndex& mi, int bb) {
    b = bb;
    const int b3 = b * b * b;
    t.assign((size_t)343 * b3, {});
    for (int uz = -3; uz <= 3; ++uz)
      for (int uy = -3; uy <= 3; ++uy)
        for (int ux = -3; ux <= 3; ++ux) {
          if (std::max(std::abs(ux), std::max(std::abs(uy), std::abs(uz))) < 2) continue;
          for (int c = 0; c < b3; ++c) {
            const int ci[3] = {c % b, (c / b) % b, c / (b * b)};
            double u[3] = {(double)ux, (double)uy, (double)uz};
            for (int q = 0; q < 3; ++q) u[q] += (ci[q] + 0.5) / b - 0.5;
            taylor_inv_r(u, mi, t[(size_t)((uz + 3) * 49 + (uy + 3) * 7 + (ux + 3)) * b3 + c]);
          }
        }
  }
};

// comps = 1: columns n = target child * b^3 + cell, the potential.  comps = 4
// (the analytic force, App. C): n = child * 4 b^3 + comp * b^3 + cell, comp 0
// the potential and comp 1 + q its derivative in the target's x_q (box
// units): d/du_q D_a(u) = D_{a + e_q}(u), and with T the Taylor coefficients
// of 1/r, D_a / a! = -T_a, so the weight is (-1)^|a| (-(a_q + 1) T_{a+e_q});
// tab then holds the coefficients to order p + 1.
double m2p_entry(const MultiIndex& mi, const M2pTable& tab, int d, int k, int n, int comps = 1) {
  const int b3 = tab.b * tab.b * tab.b;
  const int al = k / 8, cs = k % 8, ct = n / (comps * b3), comp = (n / b3) % comps, cell = n % b3;
  if (al >= mi.nc || ct >= 8 || level_of_order(mi, al) > mi.mo) return 0.0;
  const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
  int u[3];
  for (int q = 0; q < 3; ++q) u[q] = ((ct >> q) & 1) - ((cs >> q) & 1) - 2 * D[q];
  if (std::max(std::abs(u[0]), std::max(std::abs(u[1]), std::abs(u[2]))) < 2) return 0.0;
  const std::vector<double>& tb = tab.t[(size_t)((u[2] + 3) * 49 + (u[1] + 3) * 7 + (u[0] + 3)) * b3 + cell];
  const double sgn = ((mi.a[al] + mi.b[al] + mi.c[al]) & 1) ? -1.0 : 1.0;
  if (comp == 0) return sgn * (-tb[al]);
  int e[3] = {mi.a[al], mi.b[al], mi.c[al]};
  const int aq = e[comp - 1]++;
  return sgn * (-(aq + 1) * tb[mi.index(e[0], e[1], e[2])]);
}

// Tensor-core schedule of the M2P contraction: every output column needs the
// whole reduction (no truncation prefix), so groups of up to 128 columns
// share one K = 8 nc; one pass for b <= 4.
bool build_tc_m2p(const MultiIndex& mi, const M2pTable& tab, int kind, TcHost& H, bool harm, int comps = 1) {
  const int ncol = 8 * comps * tab.b * tab.b * tab.b;
  const std::vector<int> red = harmonic_components(mi);
  const int K = 8 * (harm ? (mi.mo + 1) * (mi.mo + 1) : ncoef(mi.mo));
  std::vector<TcCols> gs;
  for (int c = 0; c < ncol; c += kTcMaxGroupN) gs.push_back({c, std::min(kTcMaxGroupN, ncol - c), K});
  // with harmonic planes the reduction runs over the folded components (the
  // M2P weights, derivatives of 1/r in alpha, fold the same way)
  auto entry = [&](int d, int k, int n) {
    if (!harm) return m2p_entry(mi, tab, d, k, n, comps);
    if (k / 8 >= (int)red.size()) return 0.0;
    return m2p_entry(mi, tab, d, red[k / 8] * 8 + k % 8, n, comps);
  };
  return build_tc_generic(kind, gs, entry, H, 2);
}

// Prefix-schedule (k_nbr_tc.cu) forms of the three contractions above; they
// return false where the prefix schedule does not apply (then the span
// schedule of build_tc* runs).
bool build_tp_m2l(const MultiIndex& mi, const TaylorTable& tt, int kind, TpHost& H, bool harm) {
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  auto count = [harm](int q) { return harm ? (q + 1) * (q + 1) : ncoef(q); };
  std::vector<int> kcol(8 * nk);
  for (int n = 0; n < 8 * nk; ++n) {
    const int m = level_of_order(mi, harm ? red[n / 8] : n / 8);
    kcol[n] = 8 * count(std::min(mi.p - m, mi.mo));
  }
  auto entry = [&](int d, int k, int n) {
    if (!harm) return m2l_entry(mi, tt, d, k, n);
    return m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8);
  };
  return build_tp_generic(kind, kcol, 8 * nk, entry, H);
}

bool build_tp_near(int b, int comps, int kind, TpHost& H) {
  const int b3 = b * b * b;
  std::vector<int> kcol(comps * b3, b3);
  auto entry = [b](int d, int k, int n) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    return near_entry(b, D, k, n);
  };
  return build_tp_generic(kind, kcol, b3, entry, H);
}

bool build_tp_m2p(const MultiIndex& mi, const M2pTable& tab, int kind, TpHost& H, bool harm, int comps = 1) {
  const int ncol = 8 * comps * tab.b * tab.b * tab.b;
  const std::vector<int> red = harmonic_components(mi);
  const int K = 8 * (harm ? (mi.mo + 1) * (mi.mo + 1) : ncoef(mi.mo));
  std::vector<int> kcol(ncol, K);
  auto entry = [&](int d, int k, int n) {
    if (!harm) return m2p_entry(mi, tab, d, k, n, comps);
    if (k / 8 >= (int)red.size()) return 0.0;
    return m2p_entry(mi, tab, d, red[k / 8] * 8 + k % 8, n, comps);
  };
  return build_tp_generic(kind, kcol, K, entry, H);
}

// Weights of a CUDA-core contraction whose column tiles all reduce over K:
// W[tile][d][k][32].
template <typename T, typename Entry>
void full_weights(int ncols, int K, const Entry& entry, std::vector<T>& W, std::vector<int>& tile_k,
                  std::vector<long long>& tile_w, bool fill = true) {
  const int ntiles = (ncols + kNTile - 1) / kNTile;
  tile_k.assign(ntiles, K);
  tile_w.resize(ntiles);
  for (int t = 0; t < ntiles; ++t) tile_w[t] = 27LL * K * kNTile * t;
  W.assign((size_t)27 * K * kNTile * ntiles, T(0));
  if (!fill) return;
  for (int t = 0; t < ntiles; ++t)
    for (int d = 0; d < 27; ++d) {
      T* blk = W.data() + tile_w[t] + (long long)d * K * kNTile;
      for (int j = 0; j < kNTile; ++j) {
        const int n = t * kNTile + j;
        if (n >= ncols) continue;
        for (int k = 0; k < K; ++k) blk[(long long)k * kNTile + j] = (T)entry(d, k, n);
      }
    }
}

// Near-field matrices (eq. direct, cell units) for the CUDA-core contraction:
// W_d[s][n] = near_entry(d, s, n) for source cell s of neighbour leaf box d
// and output column n (potential, then the force components).

template <typename T>
void near_weights(int b, int comps, std::vector<T>& W, std::vector<int>& tile_k, std::vector<long long>& tile_w,
                  bool fill = true) {
  const int b3 = b * b * b;
  const int ncols = comps * b3;
  const int ntiles = (ncols + kNTile - 1) / kNTile;
  tile_k.assign(ntiles, b3);
  tile_w.resize(ntiles);
  for (int t = 0; t < ntiles; ++t) tile_w[t] = 27LL * b3 * kNTile * t;
  W.assign((size_t)27 * b3 * kNTile * ntiles, T(0));
  if (!fill) return;
  for (int t = 0; t < ntiles; ++t)
    for (int d = 0; d < 27; ++d) {
      const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
      T* blk = W.data() + tile_w[t] + (long long)d * b3 * kNTile;
      for (int j = 0; j < kNTile; ++j) {
        const int n = t * kNTile + j;
        if (n >= ncols) continue;
        for (int s = 0; s < b3; ++s) blk[(long long)s * kNTile + j] = (T)near_entry(b, D, s, n);
      }
    }
}

// M2M: Mt_alpha(P) += C(alpha,beta) 2^-|alpha| (+-1/2)^(alpha-beta) Mt_beta(C);
// L2L: Lt_beta(C) += C(gamma,beta) 2^(-1-|gamma|) (+-1/2)^(gamma-beta) Lt_gamma(P).
void shift_tables(const MultiIndex& mi, std::vector<int>& m2m_start, std::vector<ShiftEntry>& m2m,
                  std::vector<int>& l2l_start, std::vector<ShiftEntry>& l2l) {
  const int nc = mi.nc;
  m2m_start.assign(nc + 1, 0);
  l2l_start.assign(nc + 1, 0);
  m2m.clear();
  l2l.clear();
  for (int o = 0; o < nc; ++o) {
    m2m_start[o] = (int)m2m.size();
    for (int i = 0; i < nc; ++i) {
      const int d[3] = {mi.a[o] - mi.a[i], mi.b[o] - mi.b[i], mi.c[o] - mi.c[i]};
      if (d[0] < 0 || d[1] < 0 || d[2] < 0) continue;
      const int no = mi.a[o] + mi.b[o] + mi.c[o], nd = d[0] + d[1] + d[2];
      ShiftEntry e;
      e.src = i;
      e.mask = (d[0] & 1) | ((d[1] & 1) << 1) | ((d[2] & 1) << 2);
      e.coef = binom(mi.a[o], mi.a[i]) * binom(mi.b[o], mi.b[i]) * binom(mi.c[o], mi.c[i]) * std::ldexp(1.0, -no - nd);
      e.coef_f = (float)e.coef;
      m2m.push_back(e);
    }
    l2l_start[o] = (int)l2l.size();
    for (int g = 0; g < nc; ++g) {
      const int d[3] = {mi.a[g] - mi.a[o], mi.b[g] - mi.b[o], mi.c[g] - mi.c[o]};
      if (d[0] < 0 || d[1] < 0 || d[2] < 0) continue;
      const int ng = mi.a[g] + mi.b[g] + mi.c[g], nd = d[0] + d[1] + d[2];
      ShiftEntry e;
      e.src = g;
      e.mask = (d[0] & 1) | ((d[1] & 1) << 1) | ((d[2] & 1) << 2);
      e.coef = binom(mi.a[g], mi.a[o]) * binom(mi.b[g], mi.b[o]) * binom(mi.c[g], mi.c[o]) *
               std::ldexp(1.0, -1 - ng - nd);
      e.coef_f = (float)e.coef;
      l2l.push_back(e);
    }
  }
  m2m_start[nc] = (int)m2m.size();
  l2l_start[nc] = (int)l2l.size();
}

bool tc_precision(int prec) { return prec == FMM_M2L_TF32 || prec == FMM_M2L_BF16X3; }

}  // namespace

namespace {

// Everything of a plan after argument checks: hierarchy, level precisions,
// arena layout, tables.  Device memory comes from P->dev_alloc (cudaMalloc
// for plans, the static array for the allocation-free solve).  On failure
// the caller releases P.
NbrGemm m2l_gemm(fmm_plan_t P, int l);
NbrGemm near_gemm(fmm_plan_t P);

fmm_status plan_init(fmm_plan_t P, const int d3[3], double dx, double G, int order, int leaf, const fmm_opts& o,
                     cudaStream_t stream, int dev) {
  cudaStream_t s = stream;
  P->last_stream = s;
  for (int q = 0; q < 3; ++q) P->dims[q] = d3[q];
  P->dx = dx;
  P->G = G;
  P->p = order;
  P->b = leaf;
  P->opts = o;
  P->mi.init(order);
  if (o.mult_order >= 0 && o.mult_order < order) P->mi.mo = o.mult_order;
  P->nc = P->mi.nc;
  P->near_comps = o.accel == 2 ? 4 : 1;
  P->m2p = o.final_stage == 1;

  fmm_status st = build_levels(P);
  if (st != FMM_OK) return st;
  if (P->L < 2) P->m2p = false;  // no interaction list at the leaf level
  // level precisions: FP64 everywhere, FP32 everywhere, or (tensor-core
  // precisions) FP64 on the coarsest M2L levels 2 .. 1 + n_fp64_levels (never
  // the leaf level) and tcgen05 M2L on every other level.
  const bool tcp = tc_precision(o.precision);
  if (tcp) P->tc_kind = o.precision == FMM_M2L_BF16X3 ? TC_BF16X3 : TC_TF32;
  P->nr = (order + 1) * (order + 1);
  P->harm = tcp && !o.m2l_cartesian && order >= 2 && P->nr <= kTcMaxColMap;
  {
    // CUDA-core precisions only: in the mixed ones the CUDA-core (FP64) levels
    // run beside the tensor-core levels and, compressed, their denser DFMA
    // work slows those (512^3 bf16x3 step 8.35 ms against 8.11 ms).  P2M
    // stages a box row's full and folded components in shared memory.
    const size_t esz = o.precision == FMM_FP64 ? 8 : 4;
    const size_t stage = (size_t)16 * (8 * P->nc + 8 + 8 * P->nr + 8) * esz;
    P->harm_cc = (!tcp || o.coarse_fp32) && !o.m2l_cartesian && order >= 2 && stage <= 227 * 1024;
  }
  for (int l = 0; l <= P->L; ++l) {
    Level& lv = P->lev[l];
    lv.f64 = P->f64_data() ? 1 : 0;
    lv.tc = 0;
    if (tcp && l >= 2) {
      if (l <= 1 + o.n_fp64_levels && l < P->L) lv.f64 = o.coarse_fp32 ? 0 : 1;
      else lv.tc = order >= 2 ? 1 : 0;
    }
  }
  // arena
  P->lmin = P->L >= 2 ? 2 : P->L;
  size_t off = 0;
  auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
  for (int l = P->lmin; l <= P->L; ++l) {
    Level& lv = P->lev[l];
    lv.bytes = (size_t)lv.npar * 8 * P->nc * (lv.f64 ? 8 : 4);
    lv.m_off = off;
    off = align(off + lv.bytes);
    lv.l_off = off;
    off = align(off + lv.bytes);
    lv.hi_off = lv.lo_off = 0;
    lv.fold_off = lv.lred_off = 0;
    if (P->harm_cc && !lv.tc && l >= 2 && !(l == P->L && P->m2p)) {
      const size_t red = (size_t)lv.npar * 8 * P->nr * (lv.f64 ? 8 : 4);
      lv.fold_off = off;
      off = align(off + red);
      lv.lred_off = off;
      off = align(off + red);
    }
    if (P->harm && lv.tc && P->tc_kind == TC_TF32) {  // TF32 reads FP32 rows: the folded ones
      lv.fold_off = off;
      off = align(off + (size_t)lv.npar * 8 * P->nr * 4);
    }
    if (lv.tc && P->tc_kind == TC_BF16X3) {
      const size_t plane = (size_t)lv.npar * 8 * P->plane_nc() * 2;
      lv.hi_off = off;
      off = align(off + plane);
      lv.lo_off = off;
      off = align(off + plane);
    }
  }
  const size_t cells_bytes = (size_t)P->ncell() * P->esize();
  P->rho_box_off = off;
  off = align(off + cells_bytes);
  P->near_off = off;
  off = align(off + cells_bytes * (size_t)P->near_comps);
  if (P->m2p) {  // every cell of every leaf parent block, phantom children included
    P->m2p_comps = o.accel == 2 ? 4 : 1;
    P->m2p_off = off;
    off = align(off + (size_t)P->lev[P->L].npar * 8 * (size_t)(P->b * P->b * P->b) * P->m2p_comps * P->esize());
  }
  P->work_off = off;
  off = align(off + cells_bytes);
  if (P->near_comps == 4) {
    P->adj_dip_off = off;
    off = align(off + 3 * cells_bytes);
  }
  P->near_tc = tcp && (leaf == 4 || leaf == 8);
  if (P->near_tc) {  // the near field always runs bf16x3 (hi/lo density planes)
    P->rho_hi_off = off;
    off = align(off + (size_t)P->ncell() * 2);
    P->rho_lo_off = off;
    off = align(off + (size_t)P->ncell() * 2);
  }
  {
    // column tiles of the SIMT contraction (needed to size the split scratch)
    const int ncol = 8 * P->nc;
    P->m2l_ntiles = (8 * (P->harm_cc ? P->nr : P->nc) + kNTile - 1) / kNTile;
    size_t part = 0, want = 0;
    for (int l = 2; l <= P->L; ++l) {
      const size_t one = (size_t)P->lev[l].npar * (size_t)ncol * (size_t)(P->lev[l].f64 ? 8 : 4);
      if (P->split_level(l)) part = std::max(part, 27 * one);
      if (!P->lev[l].tc) want = std::max(want, 27 * one);
    }
    // room for the autotuner's neighbour-split candidates (M2L levels and the
    // near field), up to 64 MiB
    if (!P->near_tc)
      want = std::max(want, (size_t)27 * (size_t)P->lev[P->L].nbox * (size_t)(P->b * P->b * P->b) *
                                (size_t)P->near_comps * P->esize());
    if (!P->no_split) part = std::max(part, std::min(want, (size_t)64 << 20));
    P->part_off = off;
    P->part_cap = part;
    off = align(off + part);
    for (int l = 2; l <= P->L; ++l) P->m2l_choice[l].dsplit = P->split_level(l) ? 27 : 1;
  }
  // Default variants before any tuning: the small levels split over their 27
  // neighbours (4x4x4 tiles), the rest on z-run tiles where they apply.
  auto zrun_default = [&](NbrGemm g, const std::vector<int>& tk, fmm_plan_s::SimtChoice* c, bool f64) {
    g.dsplit = 1;
    if (f64 && P->tc_kind >= 0) {  // coarse FP64 levels beside the tensor-core levels
      c->shape = 3;
      return;
    }
    if (c->dsplit != 1 || !zrun_eligible(g, tk.data(), (int)tk.size())) return;
    c->shape = 1;
    // fewer than four blocks per SM: split the neighbours three ways if the
    // partial sums fit the scratch
    const long long blocks = (long long)((g.grid[0] + 7) / 8) * ((g.grid[1] + 3) / 4) * ((g.grid[2] + 7) / 8) * g.ntiles;
    const size_t part3 = (size_t)3 * g.grid[0] * g.grid[1] * g.grid[2] * (size_t)g.n_cols * (f64 ? 8 : 4);
    if (blocks < 4 * 152 && part3 <= P->part_cap) c->dsplit = 3;
  };
  P->arena_bytes = off;

  auto cleanup = [](fmm_status e) { return e; };  // the caller releases the plan
  void* arena = nullptr;
  if ((st = P->dev_alloc(P->arena_bytes, &arena))) return st;
  P->arena = static_cast<unsigned char*>(arena);
  if (!P->dry && cudaMemsetAsync(arena, 0, P->arena_bytes, s) != cudaSuccess)
    return cleanup(fail(FMM_ERR_CUDA, "memset failed"));

  // tables
  std::vector<int8_t> mi8(3 * P->nc);
  for (int k = 0; k < P->nc; ++k) {
    mi8[3 * k] = (int8_t)P->mi.a[k];
    mi8[3 * k + 1] = (int8_t)P->mi.b[k];
    mi8[3 * k + 2] = (int8_t)P->mi.c[k];
  }
  std::vector<int> m2m_start, l2l_start;
  std::vector<ShiftEntry> m2m, l2l;
  shift_tables(P->mi, m2m_start, m2m, l2l_start, l2l);
  std::vector<int> one_flag(1, 0);
  if ((st = P->upload(mi8, &P->d_mi, s)) || (st = P->upload(m2m_start, &P->d_m2m_start, s)) ||
      (st = P->upload(m2m, &P->d_m2m, s)) || (st = P->upload(l2l_start, &P->d_l2l_start, s)) ||
      (st = P->upload(l2l, &P->d_l2l, s)) || (st = P->upload(one_flag, &P->d_flag, s)))
    return cleanup(st);
  {
    bool any64 = false, any32 = false, anytc = false;
    for (int l = 2; l <= P->L; ++l) {
      any64 |= P->lev[l].f64 != 0;
      any32 |= (!P->lev[l].f64 && !P->lev[l].tc);
      anytc |= P->lev[l].tc != 0;
    }
    TaylorTable tt;
    if (P->L >= 2 && !P->static_keep_tables) tt.build(P->mi);
    std::vector<int> tk;
    std::vector<long long> tw;
    if (any64) {
      std::vector<double> W;
      m2l_weights<double>(P->mi, tt, W, tk, tw, !P->static_keep_tables, P->harm_cc);
      double* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_m2l_f64 = d;
    }
    if (any32) {
      std::vector<float> W;
      m2l_weights<float>(P->mi, tt, W, tk, tw, !P->static_keep_tables, P->harm_cc);
      float* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_m2l_f32 = d;
    }
    P->m2l_ntiles = (int)tk.size();
    P->h_m2l_tile_k = tk;
    if ((st = P->upload(tk, &P->d_m2l_tile_k, s)) || (st = P->upload(tw, &P->d_m2l_tile_w, s))) return cleanup(st);
    MultiIndex mt = P->mi;  // the transpose of a mult_order < order operator swaps the limits
    mt.mo = P->p;
    mt.lo = P->mi.mo;
    P->asym = P->mi.mo < P->p && P->L >= 2;
    if (P->asym && (any64 || any32)) {
      std::vector<int> tk2;
      std::vector<long long> tw2;
      if (any64) {
        std::vector<double> W;
        m2l_weights<double>(mt, tt, W, tk2, tw2, true, P->harm_cc);
        double* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_m2l_f64_t = d;
      }
      if (any32) {
        std::vector<float> W;
        m2l_weights<float>(mt, tt, W, tk2, tw2, true, P->harm_cc);
        float* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_m2l_f32_t = d;
      }
      if ((int)tk2.size() != P->m2l_ntiles) return cleanup(fail(FMM_ERR_CUDA, "transposed M2L tiles differ"));
      if ((st = P->upload(tk2, &P->d_m2l_tile_k_t, s)) || (st = P->upload(tw2, &P->d_m2l_tile_w_t, s)))
        return cleanup(st);
    }
    if (anytc) {
      auto fill_tp = [&](const TpHost& Hp, TpLaunch& T, const unsigned char* dw) {
        T.npass = (int)Hp.pass.size();
        for (int i = 0; i < T.npass; ++i) T.pass[i] = Hp.pass[i];
        T.a_stages = Hp.a_stages;
        T.w_slots = Hp.w_slots;
        for (int q = 0; q < kTpIssuers; ++q) T.owner_slot0[q] = (int8_t)Hp.owner_slot0[q], T.owner_nslots[q] = (int8_t)Hp.owner_nslots[q];
        T.W = dw;
        T.n_cols = 8 * P->nc;
        T.kind = P->tc_kind;
        T.accumulate = 0;
        T.col_mapped = P->harm ? 1 : 0;
        if (P->harm) {
          const std::vector<int> red = harmonic_components(P->mi);
          for (size_t r = 0; r < red.size(); ++r) T.col_map[r] = (int16_t)red[r];
        }
      };
      {
        TpHost Hp;
        if (build_tp_m2l(P->mi, tt, P->tc_kind, Hp, P->harm)) {
          unsigned char* dw = nullptr;
          if ((st = P->upload(Hp.W, &dw, s))) return cleanup(st);
          fill_tp(Hp, P->tpl, dw);
          P->tp_m2l = true;
        }
        if (P->asym) {
          TpHost Ht;
          if (build_tp_m2l(mt, tt, P->tc_kind, Ht, P->harm)) {
            unsigned char* dw = nullptr;
            if ((st = P->upload(Ht.W, &dw, s))) return cleanup(st);
            fill_tp(Ht, P->tpl_t, dw);
            P->tp_m2l_t = true;
          }
        }
      }
      TcHost H;
      P->span_m2l = build_tc(P->mi, tt, P->tc_kind, H, P->harm);
      if (!P->span_m2l) H = TcHost{};
      if (!P->span_m2l && !(P->tp_m2l && (!P->asym || P->tp_m2l_t)))
        return cleanup(fail(FMM_ERR_UNSUPPORTED, "order too high for the tensor-core schedule"));
      unsigned char* dw = nullptr;
      if (!H.W.empty() && (st = P->upload(H.W, &dw, s))) return cleanup(st);
      P->tc.W = dw;
      P->tc.npass = H.npass;
      P->tc.a_stages = H.a_stages;
      for (int i = 0; i < H.npass; ++i) P->tc.pass[i] = H.pass[i];
      P->tc.n_cols = 8 * P->nc;
      P->tc.kind = P->tc_kind;
      P->tc.col_mapped = P->harm ? 1 : 0;
      if (P->harm) {
        const std::vector<int> red = harmonic_components(P->mi);
        for (size_t r = 0; r < red.size(); ++r) P->tc.col_map[r] = (int16_t)red[r];
      }
      P->tc.err = nullptr;  // set below, after the flag exists
      TcHost Ht;
      if (P->asym) {
        P->span_m2l_t = build_tc(mt, tt, P->tc_kind, Ht, P->harm);
        if (!P->span_m2l_t && !P->tp_m2l_t)
          return cleanup(fail(FMM_ERR_UNSUPPORTED, "order too high for the transposed tensor-core schedule"));
      }
      if (P->asym && P->span_m2l_t) {
        unsigned char* dwt = nullptr;
        if ((st = P->upload(Ht.W, &dwt, s))) return cleanup(st);
        P->tc_t = P->tc;  // same maps, columns and kind; its own passes and weights
        P->tc_t.W = dwt;
        P->tc_t.npass = Ht.npass;
        P->tc_t.a_stages = Ht.a_stages;
        for (int i = 0; i < Ht.npass; ++i) P->tc_t.pass[i] = Ht.pass[i];
      }
      for (int l = 2; l <= P->L; ++l) {
        const Level& lv = P->lev[l];
        if (!lv.tc) continue;
        cudaError_t e;
        if (P->tc_kind == TC_BF16X3) {
          e = make_row_map(P->map_hi[l], P->arena + lv.hi_off, 8 * P->plane_nc(), 2, lv.np, 64);
          if (e == cudaSuccess)
            e = make_row_map(P->map_lo[l], P->arena + lv.lo_off, 8 * P->plane_nc(), 2, lv.np, 64);
        } else {
          e = lv.fold_off ? make_row_map(P->map_hi[l], P->arena + lv.fold_off, 8 * P->nr, 4, lv.np, 32)
                          : make_row_map(P->map_hi[l], P->arena + lv.m_off, 8 * P->nc, 4, lv.np, 32);
          if (e == cudaSuccess) std::memcpy(P->map_lo[l], P->map_hi[l], 128);
        }
        if (e != cudaSuccess) return cleanup(fail(FMM_ERR_CUDA, "tensor map encoding failed for level %d", l));
      }
    }
  }
  {
    std::vector<int> tk;
    std::vector<long long> tw;
    if (P->f64_data()) {
      std::vector<double> W;
      near_weights<double>(P->b, P->near_comps, W, tk, tw, !P->static_keep_tables);
      double* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_near = d;
    } else {
      std::vector<float> W;
      near_weights<float>(P->b, P->near_comps, W, tk, tw, !P->static_keep_tables);
      float* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_near = d;
    }
    P->near_ntiles = (int)tk.size();
    P->h_near_tile_k = tk;
    if ((st = P->upload(tk, &P->d_near_tile_k, s)) || (st = P->upload(tw, &P->d_near_tile_w, s))) return cleanup(st);
  }
  if (P->near_comps == 4) {
    // the near field (potential and pair forces) transposed: row box = source
    // box, reduction k = (input column, cell of neighbour box d), output the
    // source cell's potential column.  Column 0: the symmetric kernel; column
    // 1 + q: the forward force at the neighbour's cell (the target) from this
    // cell, near_entry with the opposite box offset.
    const int b = P->b, b3 = b * b * b;
    auto entry = [b, b3](int d, int k, int n) {
      const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1}, Dm[3] = {-D[0], -D[1], -D[2]};
      const int comp = k / b3, cell = k % b3;
      return comp == 0 ? near_entry(b, D, cell, n) : near_entry(b, Dm, n, comp * b3 + cell);
    };
    std::vector<int> tk;
    std::vector<long long> tw;
    if (P->f64_data()) {
      std::vector<double> W;
      full_weights<double>(b3, 4 * b3, entry, W, tk, tw, !P->static_keep_tables);
      double* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_near_adj = d;
    } else {
      std::vector<float> W;
      full_weights<float>(b3, 4 * b3, entry, W, tk, tw, !P->static_keep_tables);
      float* d = nullptr;
      if ((st = P->upload(W, &d, s))) return cleanup(st);
      P->d_w_near_adj = d;
    }
    P->near_adj_ntiles = (int)tk.size();
    P->h_near_adj_tile_k = tk;
    if ((st = P->upload(tk, &P->d_near_adj_tile_k, s)) || (st = P->upload(tw, &P->d_near_adj_tile_w, s)))
      return cleanup(st);
  }
  if (P->m2p) {
    const int mc = P->m2p_comps;
    M2pTable tab;  // Taylor coefficients to order p + 1 when the force needs the derivatives
    {
      MultiIndex mt1;
      mt1.init(P->mi.p + (mc > 1 ? 1 : 0));
      tab.build(mt1, P->b);
    }
    const Level& lf = P->lev[P->L];
    if (lf.tc) {
      TpHost Hp;
      if (build_tp_m2p(P->mi, tab, P->tc_kind, Hp, P->harm, mc)) {
        unsigned char* dw = nullptr;
        if ((st = P->upload(Hp.W, &dw, s))) return cleanup(st);
        TpLaunch& T = P->tpm;
        T.npass = (int)Hp.pass.size();
        for (int i = 0; i < T.npass; ++i) T.pass[i] = Hp.pass[i];
        T.a_stages = Hp.a_stages;
        T.w_slots = Hp.w_slots;
        for (int q = 0; q < kTpIssuers; ++q) T.owner_slot0[q] = (int8_t)Hp.owner_slot0[q], T.owner_nslots[q] = (int8_t)Hp.owner_nslots[q];
        T.W = dw;
        T.n_cols = 8 * mc * P->b * P->b * P->b;
        T.kind = P->tc_kind;
        T.accumulate = 0;
        for (int q = 0; q < 3; ++q) T.grid[q] = lf.np[q];
        T.C = reinterpret_cast<float*>(P->arena + P->m2p_off);
        P->tp_m2p = P->m2p_tc = true;
      }
    }
    if (lf.tc) {
      TcHost H;
      if (build_tc_m2p(P->mi, tab, P->tc_kind, H, P->harm, mc) && H.npass <= kTcMaxPasses) {
        unsigned char* dw = nullptr;
        if ((st = P->upload(H.W, &dw, s))) return cleanup(st);
        TcLaunch& T = P->tcm;
        T.W = dw;
        T.npass = H.npass;
        T.a_stages = H.a_stages;
        for (int i = 0; i < H.npass; ++i) T.pass[i] = H.pass[i];
        T.n_cols = 8 * mc * P->b * P->b * P->b;
        T.kind = P->tc_kind;
        T.accumulate = 0;
        for (int q = 0; q < 3; ++q) T.grid[q] = lf.np[q];
        T.C = reinterpret_cast<float*>(P->arena + P->m2p_off);
        P->m2p_tc = P->span_m2p = true;
      }
    }
    if (!P->m2p_tc) {
      const int ncol = 8 * mc * P->b * P->b * P->b;
      auto entry = [&](int d, int k, int n) { return m2p_entry(P->mi, tab, d, k, n, mc); };
      std::vector<int> tk;
      std::vector<long long> tw;
      if (lf.f64) {
        std::vector<double> W;
        full_weights<double>(ncol, 8 * ncoef(P->mi.mo), entry, W, tk, tw);
        double* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_m2p = d;
      } else {
        std::vector<float> W;
        full_weights<float>(ncol, 8 * ncoef(P->mi.mo), entry, W, tk, tw);
        float* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_m2p = d;
      }
      P->m2p_ntiles = (int)tk.size();
      P->h_m2p_tile_k = tk;
      if ((st = P->upload(tk, &P->d_m2p_tile_k, s)) || (st = P->upload(tw, &P->d_m2p_tile_w, s))) return cleanup(st);
    }
    {
      // P2L = M2P transposed: rows are source parents, the reduction runs over
      // the cells (target child, cell) of neighbour d, the columns are the
      // source's (alpha, child) locals; W'_d[k][n] = W_{-d}[n][k] (26 - d is
      // the opposite neighbour)
      const int K = 8 * mc * P->b * P->b * P->b;
      auto entry = [&](int d, int k, int n) { return m2p_entry(P->mi, tab, 26 - d, n, k, mc); };
      std::vector<int> tk;
      std::vector<long long> tw;
      if (lf.f64) {
        std::vector<double> W;
        full_weights<double>(8 * P->nc, K, entry, W, tk, tw);
        double* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_p2l = d;
      } else {
        std::vector<float> W;
        full_weights<float>(8 * P->nc, K, entry, W, tk, tw);
        float* d = nullptr;
        if ((st = P->upload(W, &d, s))) return cleanup(st);
        P->d_w_p2l = d;
      }
      P->p2l_ntiles = (int)tk.size();
      P->h_p2l_tile_k = tk;
      if ((st = P->upload(tk, &P->d_p2l_tile_k, s)) || (st = P->upload(tw, &P->d_p2l_tile_w, s))) return cleanup(st);
    }
  }
  if (P->near_tc) {
    TpHost Hp;
    if (build_tp_near(P->b, P->near_comps, TC_BF16X3, Hp)) {
      unsigned char* dw = nullptr;
      if ((st = P->upload(Hp.W, &dw, s))) return cleanup(st);
      TpLaunch& T = P->tpn;
      T.npass = (int)Hp.pass.size();
      for (int i = 0; i < T.npass; ++i) T.pass[i] = Hp.pass[i];
      T.a_stages = Hp.a_stages;
      T.w_slots = Hp.w_slots;
      for (int q = 0; q < kTpIssuers; ++q) T.owner_slot0[q] = (int8_t)Hp.owner_slot0[q], T.owner_nslots[q] = (int8_t)Hp.owner_nslots[q];
      T.W = dw;
      T.n_cols = P->b * P->b * P->b * P->near_comps;
      T.kind = TC_BF16X3;
      T.accumulate = 0;
      for (int q = 0; q < 3; ++q) T.grid[q] = P->lev[P->L].n[q];
      T.C = reinterpret_cast<float*>(P->arena + P->near_off);
      P->tp_near = true;
    }
  }
  if (P->near_tc) {
    TcHost H;
    // bf16x3 in both tensor-core precisions: a TF32 near field would carry
    // ~3e-4 relative error on its (same-signed) sums
    P->span_near = build_tc_near(P->b, P->near_comps, TC_BF16X3, H);
    if (!P->span_near && !P->tp_near) return cleanup(fail(FMM_ERR_UNSUPPORTED, "near-field schedule failed"));
    if (P->span_near) {
      unsigned char* dw = nullptr;
      if ((st = P->upload(H.W, &dw, s))) return cleanup(st);
      // every launch writes its own columns of the same rows
      P->tcn.assign((H.npass + kTcMaxPasses - 1) / kTcMaxPasses, TcLaunch{});
      for (size_t li = 0; li < P->tcn.size(); ++li) {
        TcLaunch& T = P->tcn[li];
        T.W = dw;
        T.npass = std::min(kTcMaxPasses, H.npass - (int)li * kTcMaxPasses);
        T.a_stages = H.a_stages;
        for (int i = 0; i < T.npass; ++i) T.pass[i] = H.pass[li * kTcMaxPasses + i];
        T.n_cols = P->b * P->b * P->b * P->near_comps;
        T.kind = TC_BF16X3;
        T.accumulate = 0;
        for (int q = 0; q < 3; ++q) T.grid[q] = P->lev[P->L].n[q];
        T.C = reinterpret_cast<float*>(P->arena + P->near_off);
        T.err = P->d_flag;
      }
    }
  }
  if (P->near_tc && P->b == 4 && P->near_comps == 1) {
    std::vector<unsigned char> W4;
    near4_weights(W4);
    unsigned char* dw = nullptr;
    if ((st = P->upload(W4, &dw, s))) return cleanup(st);
    P->ntl.W = dw;
    P->ntl.C = reinterpret_cast<float*>(P->arena + P->near_off);
    for (int q = 0; q < 3; ++q) P->ntl.grid[q] = P->lev[P->L].n[q];
    P->ntl.err = P->d_flag;
    P->ntl.idesc = host_idesc(TC_BF16X3, 64);
    P->near4 = true;
  }
  if (P->near_tc) {
    // activation rows: the b^3 cell values of a leaf box (the output rows carry
    // near_comps x b^3 columns)
    const int b3 = P->b * P->b * P->b;
    const int* ng = P->lev[P->L].n;
    cudaError_t e = make_row_map(P->map_near_hi, P->arena + P->rho_hi_off, b3, 2, ng, 64);
    if (e == cudaSuccess) e = make_row_map(P->map_near_lo, P->arena + P->rho_lo_off, b3, 2, ng, 64);
    if (e != cudaSuccess) return cleanup(fail(FMM_ERR_CUDA, "tensor map encoding failed for the near field"));
  }
  P->tpl.err = P->tpl_t.err = P->tpm.err = P->tpn.err = P->d_flag;
  P->tc.err = P->d_flag;
  P->tc.accumulate = 0;
  P->tc_t.err = P->d_flag;
  P->tc_t.accumulate = 0;
  P->tcm.err = P->d_flag;
  for (int l = 2; l <= P->L; ++l)
    if (!P->lev[l].tc) zrun_default(m2l_gemm(P, l), P->h_m2l_tile_k, &P->m2l_choice[l], P->lev[l].f64);
  if (!P->near_tc) zrun_default(near_gemm(P), P->h_near_tile_k, &P->near_choice, P->f64_data());
  // uploads read host vectors that go out of scope here (plans only; the
  // allocation-free solve orders its copies on the caller's stream)
  if (!P->static_base && cudaStreamSynchronize(s) != cudaSuccess)
    return cleanup(fail(FMM_ERR_CUDA, "table upload failed"));
  return FMM_OK;
}

}  // namespace

extern "C" {

void fmm_default_opts(fmm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FMM_FP32;
  o->n_fp64_levels = 3;
  o->accel = 1;
  o->mult_order = -1;
  o->coarse_fp32 = 1;
}

const char* fmm_last_error(void) { return g_last_error.c_str(); }

// The side stream (CUDA-core M2L levels) gets the highest priority: its few
// small blocks are then scheduled ahead of queued tensor-core blocks and
// finish early instead of trickling through the whole far-field phase.
static int side_priority() {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
  return greatest;
}

fmm_status fmm_plan(const fmm_grid* grid, int order, int leaf, const fmm_opts* opts, void* stream, fmm_plan_t* out) {
  g_last_error.clear();
  if (!out) return fail(FMM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid) return fail(FMM_ERR_ARG, "grid is NULL");
  if (order < 0 || order > kMaxOrder) return fail(FMM_ERR_ARG, "order %d outside [0, %d]", order, kMaxOrder);
  if (leaf != 2 && leaf != 4 && leaf != 8) return fail(FMM_ERR_ARG, "leaf %d not in {2, 4, 8}", leaf);
  const int d3[3] = {grid->nx, grid->ny, grid->nz};
  for (int q = 0; q < 3; ++q) {
    if (d3[q] <= 0) return fail(FMM_ERR_ARG, "grid extent %d must be positive", d3[q]);
    if (d3[q] % leaf) return fail(FMM_ERR_ARG, "grid extent %d is not a multiple of leaf %d", d3[q], leaf);
    if (d3[q] > (1 << 14)) return fail(FMM_ERR_ARG, "grid extent %d too large", d3[q]);
  }
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx)) return fail(FMM_ERR_ARG, "dx must be positive and finite");
  if (!std::isfinite(grid->G)) return fail(FMM_ERR_ARG, "G must be finite");
  fmm_opts o;
  if (opts) {
    o = *opts;
  } else {
    fmm_default_opts(&o);
  }
  if (o.precision < FMM_FP64 || o.precision > FMM_M2L_BF16X3) return fail(FMM_ERR_ARG, "unknown precision %d", o.precision);
  if (o.n_fp64_levels < 0 || o.n_fp64_levels > kMaxLevels) return fail(FMM_ERR_ARG, "bad n_fp64_levels");
  if (o.accel < 0 || o.accel > 2) return fail(FMM_ERR_ARG, "accel %d not in {0, 1, 2}", o.accel);
  if (o.final_stage < 0 || o.final_stage > 1) return fail(FMM_ERR_ARG, "final_stage %d not in {0, 1}", o.final_stage);
  if (o.m2l_cartesian < 0 || o.m2l_cartesian > 1) return fail(FMM_ERR_ARG, "m2l_cartesian %d not in {0, 1}", o.m2l_cartesian);
  if (o.mult_order < -1) return fail(FMM_ERR_ARG, "mult_order %d below -1", o.mult_order);
  if (o.coarse_fp32 < 0 || o.coarse_fp32 > 1) return fail(FMM_ERR_ARG, "coarse_fp32 %d not in {0, 1}", o.coarse_fp32);
  for (int r : o.reserved)
    if (r != 0) return fail(FMM_ERR_ARG, "reserved option fields must be zero");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (tc_precision(o.precision)) {
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3))
      return fail(FMM_ERR_UNSUPPORTED, "tensor-core precisions need an sm_103 device (found sm_%d%d)", prop.major,
                  prop.minor);
  }

  fmm_plan_t P = new (std::nothrow) fmm_plan_s();
  if (!P) return fail(FMM_ERR_ALLOC, "host allocation failed");
  fmm_status st = plan_init(P, d3, grid->dx, grid->G, order, leaf, o, static_cast<cudaStream_t>(stream), dev);
  if (st == FMM_OK &&
      (cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, side_priority()) != cudaSuccess ||
       cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess))
    st = fail(FMM_ERR_CUDA, "stream or event creation failed");
  if (st != FMM_OK) {
    P->release();
    delete P;
    return st;
  }
  *out = P;
  return FMM_OK;
}

}  // extern "C"

namespace {

// Records a pair of events around one stage when timing is enabled.
struct StageTimer {
  fmm_plan_t P;
  int stage;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  StageTimer(fmm_plan_t P_, int stage_, cudaStream_t s_) : P(P_), stage(stage_), s(s_) {
    if (P->timing && P->ev_used + 2 <= P->ev_pool.size()) {
      cudaEvent_t a = P->ev_pool[P->ev_used++];
      b = P->ev_pool[P->ev_used++];
      cudaEventRecord(a, s);
      P->recs.push_back({stage, a, b});
    }
  }
  ~StageTimer() {
    if (b) cudaEventRecord(b, s);
  }
};

// The last L2L (L - 1 -> leaf) runs inside the leaf kernel (potential-only
// near field, M2L final stage, both levels in the data's type); the leaf
// level's locals then stay the M2L's in memory.
bool fused_down(fmm_plan_t P) {
  const int L = P->L;
  if (L < 3 || P->m2p || P->near_comps != 1) return false;
  const int want = P->f64_data() ? 1 : 0;
  return P->lev[L].f64 == want && P->lev[L - 1].f64 == want;
}

// Per-level dispatch helpers (a level's expansions are FP64 or FP32).
fmm_status do_m2m(fmm_plan_t P, const TreeTables& tt, int l, cudaStream_t s) {
  const Level &c = P->lev[l], &q = P->lev[l - 1];
  const bool planes = q.tc && P->tc_kind == TC_BF16X3;
  void* hi = planes ? P->arena + q.hi_off : nullptr;
  void* lo = planes ? P->arena + q.lo_off : nullptr;
  void* fold = q.fold_off ? P->arena + q.fold_off : nullptr;
  const int harm = (planes && P->harm) || fold ? 1 : 0;
  cudaError_t e;
  if (c.f64)
    e = launch_m2m<double, double>(tt, c, static_cast<const double*>(P->M(l)), q, static_cast<double*>(P->M(l - 1)),
                                   nullptr, nullptr, harm, static_cast<double*>(fold), s);
  else if (q.f64)
    e = launch_m2m<float, double>(tt, c, static_cast<const float*>(P->M(l)), q, static_cast<double*>(P->M(l - 1)),
                                  nullptr, nullptr, harm, static_cast<double*>(fold), s);
  else
    e = launch_m2m<float, float>(tt, c, static_cast<const float*>(P->M(l)), q, static_cast<float*>(P->M(l - 1)), hi,
                                 lo, harm, static_cast<float*>(fold), s);
  CUDA_TRY(e);
  return FMM_OK;
}

// L(l) += L2L(L(l - 1)) for l >= 3; the level's M2L has written L(l) (level 2
// has no parent far field: its locals are its M2L alone).
// A harmonic tensor-core M2L wrote only the c <= 1 locals: L2L rebuilds the
// rest first.  l == 2 (no parent far field) with a harmonic M2L: the rebuild
// alone (no parent locals).
bool harmonic_m2l_level(fmm_plan_t P, int l) {
  return ((P->harm && P->lev[l].tc) || P->lev[l].lred_off) && !(l == P->L && P->m2p);
}

fmm_status do_l2l(fmm_plan_t P, const TreeTables& tt, int l, cudaStream_t s, int accumulate) {
  const Level &q = P->lev[l - 1], &c = P->lev[l];
  const int harm = accumulate && harmonic_m2l_level(P, l) ? 1 : 0;
  const void* red = harm && c.lred_off ? P->arena + c.lred_off : nullptr;  // CUDA-core harmonic: compact rows
  cudaError_t e;
  if (l == 2 && c.f64) {
    e = launch_l2l<double, double>(tt, q, nullptr, c, static_cast<double*>(P->Lx(l)), 1, harm,
                                   static_cast<const double*>(red), s);
  } else if (l == 2) {
    e = launch_l2l<float, float>(tt, q, nullptr, c, static_cast<float*>(P->Lx(l)), 1, harm,
                                 static_cast<const float*>(red), s);
  } else if (q.f64 && c.f64) {
    e = launch_l2l<double, double>(tt, q, static_cast<const double*>(P->Lx(l - 1)), c, static_cast<double*>(P->Lx(l)),
                                   accumulate, harm, static_cast<const double*>(red), s);
  } else if (q.f64) {
    e = launch_l2l<double, float>(tt, q, static_cast<const double*>(P->Lx(l - 1)), c, static_cast<float*>(P->Lx(l)),
                                  accumulate, harm, static_cast<const float*>(red), s);
  } else {
    e = launch_l2l<float, float>(tt, q, static_cast<const float*>(P->Lx(l - 1)), c, static_cast<float*>(P->Lx(l)),
                                 accumulate, harm, static_cast<const float*>(red), s);
  }
  CUDA_TRY(e);
  return FMM_OK;
}

NbrGemm m2l_gemm(fmm_plan_t P, int l) {
  const Level& lv = P->lev[l];
  NbrGemm g;
  // harmonic: folded multipoles in, the c <= 1 locals out (compact rows)
  const int nk = lv.fold_off ? P->nr : P->nc;
  g.A = lv.fold_off ? static_cast<void*>(P->arena + lv.fold_off) : P->M(l);
  g.row_len = 8 * nk;
  for (int q = 0; q < 3; ++q) g.grid[q] = lv.np[q];
  const bool tr = P->transposed && P->asym;
  g.W = lv.f64 ? (tr ? P->d_w_m2l_f64_t : P->d_w_m2l_f64) : (tr ? P->d_w_m2l_f32_t : P->d_w_m2l_f32);
  g.tile_k = tr ? P->d_m2l_tile_k_t : P->d_m2l_tile_k;
  g.tile_w = tr ? P->d_m2l_tile_w_t : P->d_m2l_tile_w;
  g.C = lv.lred_off ? static_cast<void*>(P->arena + lv.lred_off) : P->Lx(l);
  g.n_cols = 8 * nk;
  g.ntiles = P->m2l_ntiles;
  g.accumulate = 0;  // M2L writes the level's locals; L2L adds the parent's
  g.shape = P->m2l_choice[l].shape;
  g.dsplit = P->m2l_choice[l].dsplit;
  g.partial = P->arena + P->part_off;
  g.skip_center = 1;  // the interaction list holds no child of the same parent
  return g;
}

NbrGemm near_gemm(fmm_plan_t P) {
  NbrGemm g;
  g.A = P->arena + P->rho_box_off;
  g.row_len = P->b * P->b * P->b;
  for (int q = 0; q < 3; ++q) g.grid[q] = P->lev[P->L].n[q];
  g.W = P->d_w_near;
  g.tile_k = P->d_near_tile_k;
  g.tile_w = P->d_near_tile_w;
  g.C = P->arena + P->near_off;
  g.n_cols = P->b * P->b * P->b * P->near_comps;
  g.ntiles = P->near_ntiles;
  g.accumulate = 0;
  g.shape = P->near_choice.shape;
  g.dsplit = P->near_choice.dsplit;
  g.partial = P->arena + P->part_off;
  return g;
}

// Which tensor-core schedule a contraction runs: the prefix form when it is
// the only one, or when both exist and it is selected.
enum TcSched { TS_M2L = 0, TS_NEAR = 1, TS_M2P = 2 };
bool tc_prefix(fmm_plan_t P, int what) {
  const bool tp = what == TS_M2L ? ((P->transposed && P->asym) ? P->tp_m2l_t : P->tp_m2l)
                                 : what == TS_NEAR ? P->tp_near : P->tp_m2p;
  const bool span = what == TS_M2L ? ((P->transposed && P->asym) ? P->span_m2l_t : P->span_m2l)
                                   : what == TS_NEAR ? P->span_near : P->span_m2p;
  return tp && (P->use_tp[what] || !span);
}

// Tensor-core near field: the dedicated leaf-4 kernel, or the prefix or span
// schedule.
fmm_status do_near_tc(fmm_plan_t P, cudaStream_t s) {
  if (P->near4 && P->use_near4) {
    CUDA_TRY(launch_near_tc4(P->ntl, P->map_near_hi, P->map_near_lo, s));
  } else if (tc_prefix(P, TS_NEAR)) {
    CUDA_TRY(launch_nbr_tc(P->tpn, P->map_near_hi, P->map_near_lo, s));
  } else {
    for (const TcLaunch& NL : P->tcn) CUDA_TRY(launch_m2l_tc(NL, P->map_near_hi, P->map_near_lo, s));
  }
  return FMM_OK;
}

// Final-stage M2P of the leaf level (tensor cores when the leaf level is on
// them and the schedule fits, else the CUDA-core contraction).
fmm_status do_m2p(fmm_plan_t P, cudaStream_t s) {
  const Level& lf = P->lev[P->L];
  if (tc_prefix(P, TS_M2P)) {
    CUDA_TRY(launch_nbr_tc(P->tpm, P->map_hi[P->L], P->map_lo[P->L], s));
    return FMM_OK;
  }
  if (P->m2p_tc) {
    CUDA_TRY(launch_m2l_tc(P->tcm, P->map_hi[P->L], P->map_lo[P->L], s));
    return FMM_OK;
  }
  NbrGemm g;
  g.A = P->M(P->L);
  g.row_len = 8 * P->nc;
  for (int q = 0; q < 3; ++q) g.grid[q] = lf.np[q];
  g.W = P->d_w_m2p;
  g.tile_k = P->d_m2p_tile_k;
  g.tile_w = P->d_m2p_tile_w;
  g.C = P->arena + P->m2p_off;
  g.n_cols = 8 * P->m2p_comps * P->b * P->b * P->b;
  g.ntiles = P->m2p_ntiles;
  g.accumulate = 0;
  g.dsplit = 1;
  g.partial = nullptr;
  g.shape = zrun_eligible(g, P->h_m2p_tile_k.data(), P->m2p_ntiles) ? 1 : 0;
  CUDA_TRY(lf.f64 ? launch_nbr_gemm<double>(g, s) : launch_nbr_gemm<float>(g, s));
  return FMM_OK;
}

// Adjoint of the final-stage M2P: the leaf locals from the adjoint source's
// cells (parent-blocked in the M2P buffer), L2P then evaluates them.
fmm_status do_p2l(fmm_plan_t P, cudaStream_t s) {
  const Level& lf = P->lev[P->L];
  NbrGemm g;
  g.A = P->arena + P->m2p_off;
  g.row_len = 8 * P->m2p_comps * P->b * P->b * P->b;
  for (int q = 0; q < 3; ++q) g.grid[q] = lf.np[q];
  g.W = P->d_w_p2l;
  g.tile_k = P->d_p2l_tile_k;
  g.tile_w = P->d_p2l_tile_w;
  g.C = P->Lx(P->L);
  g.n_cols = 8 * P->nc;
  g.ntiles = P->p2l_ntiles;
  g.accumulate = 0;
  g.dsplit = 1;
  g.partial = nullptr;
  g.shape = zrun_eligible(g, P->h_p2l_tile_k.data(), P->p2l_ntiles) ? 1 : 0;
  CUDA_TRY(lf.f64 ? launch_nbr_gemm<double>(g, s) : launch_nbr_gemm<float>(g, s));
  return FMM_OK;
}

fmm_status do_m2l(fmm_plan_t P, int l, cudaStream_t s) {
  const Level& lv = P->lev[l];
  if (lv.tc && tc_prefix(P, TS_M2L)) {
    TpLaunch& L = (P->transposed && P->asym) ? P->tpl_t : P->tpl;
    L.C = static_cast<float*>(P->Lx(l));
    for (int q = 0; q < 3; ++q) L.grid[q] = lv.np[q];
    L.skip_first_a = P->inject_timeout ? 1 : 0;
    P->inject_timeout = false;
    const cudaError_t e = launch_nbr_tc(L, P->map_hi[l], P->map_lo[l], s);
    L.skip_first_a = 0;
    CUDA_TRY(e);
    return FMM_OK;
  }
  if (lv.tc) {
    TcLaunch L = (P->transposed && P->asym) ? P->tc_t : P->tc;
    L.C = static_cast<float*>(P->Lx(l));
    for (int q = 0; q < 3; ++q) L.grid[q] = lv.np[q];
    CUDA_TRY(launch_m2l_tc(L, P->map_hi[l], P->map_lo[l], s));
    return FMM_OK;
  }
  const NbrGemm g = m2l_gemm(P, l);
  CUDA_TRY(lv.f64 ? launch_nbr_gemm<double>(g, s) : launch_nbr_gemm<float>(g, s));
  return FMM_OK;
}

// adjoint = true (fmm_solve_adjoint): the same chain on the adjoint source,
// except that with the final-stage M2P the leaf level runs its transpose
// (P2L into the leaf locals, then L2L adds the parents' and L2P evaluates);
// the coarser levels and the near field are symmetric.
template <typename T>
fmm_status run_solve(fmm_plan_t P, const T* rho, T* phi, T* accel, cudaStream_t s, bool adjoint = false) {
  const TreeTables tt = P->tables();
  const int L = P->L;
  T* rho_box = reinterpret_cast<T*>(P->arena + P->rho_box_off);
  T* near_box = reinterpret_cast<T*>(P->arena + P->near_off);
  fmm_status st;
  // The transpose of the analytic force (adjoint solve with its input g):
  // with v = -g / (dx b) its far part is dipole sources in the P2M (and the
  // P2L's three force columns); its near part and the potential's are one
  // contraction over [w, -g/dx] per box, whose single output column replaces
  // the near field (the leaf finish scales both by G dx^2, as -G dx / b^2 /
  // (G dx^2 / b) = -1 / (dx b) and -G dx / (G dx^2) = -1/dx make them the
  // force's transpose).
  const T* adj_g = adjoint ? static_cast<const T*>(P->adj_g) : nullptr;
  T* adj_dip = adj_g ? reinterpret_cast<T*>(P->arena + P->adj_dip_off) : nullptr;
  if (adj_g) CUDA_TRY(launch_scaled_copy<T>(adj_g, 3 * P->ncell(), -1.0 / (P->dx * P->b), adj_dip, s));
  // upward pass
  {
    StageTimer t(P, ST_P2M, s);
    const Level& lf = P->lev[L];
    const bool mplanes = lf.tc && P->tc_kind == TC_BF16X3;
    const bool near_rows = !adj_g;  // the near field's own inputs (not read by the transposed force's)
    CUDA_TRY(launch_p2m<T>(tt, rho, P->dims, lf, static_cast<T*>(P->M(L)),
                           (P->near_tc || !near_rows) ? nullptr : rho_box,
                           mplanes ? P->arena + lf.hi_off : nullptr, mplanes ? P->arena + lf.lo_off : nullptr,
                           (P->near_tc && near_rows) ? P->arena + P->rho_hi_off : nullptr,
                           (P->near_tc && near_rows) ? P->arena + P->rho_lo_off : nullptr, P->d_flag,
                           ((mplanes && P->harm) || lf.fold_off) ? 1 : 0,
                           lf.fold_off ? reinterpret_cast<T*>(P->arena + lf.fold_off) : nullptr, s, adj_dip));
  }
  const bool p2l = adjoint && P->m2p;  // leaf level by the transpose of M2P
  if (p2l && P->m2p_comps == 4)  // [w, v] per box, the force columns zero without g
    CUDA_TRY(launch_cells_to_boxes4<T>(rho, adj_g, -1.0 / (P->dx * P->b), P->dims, P->lev[L], P->b, 1,
                                       reinterpret_cast<T*>(P->arena + P->m2p_off), s));
  else if (p2l)
    CUDA_TRY(launch_cells_to_parent_blocks<T>(rho, P->dims, P->lev[L], P->b,
                                              reinterpret_cast<T*>(P->arena + P->m2p_off), s));
  for (int l = L; l >= 3; --l) {
    StageTimer t(P, ST_M2M, s);
    if ((st = do_m2m(P, tt, l, s))) return st;
  }
  // Far and near field.  Each level's M2L reads only the multipoles, so all
  // levels run at once: the CUDA-core levels (FP64 coarse levels, or every
  // level of the FP32/FP64 precisions) on the plan's side stream, the
  // tensor-core levels and the near field on `s`; the two use different
  // units of the SM.  The L2L chain then adds the parents' locals, coarse to
  // fine.  A near field split over neighbour groups shares the split scratch
  // with the CUDA-core levels, so it runs after them on the same stream.
  if (L < 2) {
    StageTimer t(P, ST_L2L, s);
    CUDA_TRY(launch_zero<T>(static_cast<T*>(P->Lx(L)), P->lev[L].bytes / sizeof(T), s));
  }
  bool any_simt = false;
  for (int l = 2; l <= L; ++l) any_simt |= !P->lev[l].tc;
  const bool near_side = !P->near_tc && P->near_choice.dsplit > 1 && !adj_g;
  const bool fork = P->side && (any_simt || near_side);
  cudaStream_t sf = fork ? P->side : s;
  if (fork) {
    CUDA_TRY(cudaEventRecord(P->ev_fork, s));
    CUDA_TRY(cudaStreamWaitEvent(sf, P->ev_fork, 0));
  }
  for (int l = 2; l <= L; ++l) {
    if (P->lev[l].tc || (p2l && l == L)) continue;
    StageTimer t(P, ST_M2L, sf);
    if ((st = (l == L && P->m2p) ? do_m2p(P, sf) : do_m2l(P, l, sf))) return st;
  }
  if (p2l) {
    StageTimer t(P, ST_M2L, sf);
    if ((st = do_p2l(P, sf))) return st;
  }
  if (near_side) {
    StageTimer t(P, ST_NEAR, sf);
    CUDA_TRY(launch_nbr_gemm<T>(near_gemm(P), sf));
  }
  if (fork) CUDA_TRY(cudaEventRecord(P->ev_join, sf));
  for (int l = 2; l <= L; ++l) {
    if (!P->lev[l].tc || (p2l && l == L)) continue;
    StageTimer t(P, ST_M2L_TC, s);
    if ((st = (l == L && P->m2p) ? do_m2p(P, s) : do_m2l(P, l, s))) return st;
  }
  // near field over the 27 neighbour leaf boxes
  if (adj_g) {  // the transposed near field of the potential and the force, one output column
    StageTimer t(P, ST_NEAR, s);
    CUDA_TRY(launch_cells_to_boxes4<T>(rho, adj_g, -1.0 / P->dx, P->dims, P->lev[L], P->b, 0, near_box, s));
    NbrGemm g;
    g.A = near_box;
    g.row_len = 4 * P->b * P->b * P->b;
    for (int q = 0; q < 3; ++q) g.grid[q] = P->lev[L].n[q];
    g.W = P->d_w_near_adj;
    g.tile_k = P->d_near_adj_tile_k;
    g.tile_w = P->d_near_adj_tile_w;
    g.C = rho_box;
    g.n_cols = P->b * P->b * P->b;
    g.ntiles = P->near_adj_ntiles;
    g.accumulate = 0;
    g.dsplit = 1;
    g.partial = nullptr;
    g.shape = zrun_eligible(g, P->h_near_adj_tile_k.data(), P->near_adj_ntiles) ? 1 : 0;
    CUDA_TRY(launch_nbr_gemm<T>(g, s));
  } else if (P->near_tc) {
    StageTimer t(P, ST_NEAR_TC, s);
    if ((st = do_near_tc(P, s))) return st;
  } else if (!near_side) {
    StageTimer t(P, ST_NEAR, s);
    CUDA_TRY(launch_nbr_gemm<T>(near_gemm(P), s));
  }
  if (fork) CUDA_TRY(cudaStreamWaitEvent(s, P->ev_join, 0));
  if (L >= 2 && harmonic_m2l_level(P, 2)) {  // level 2 locals are its M2L alone: rebuild
    StageTimer t(P, ST_L2L, s);
    if ((st = do_l2l(P, tt, 2, s, 1))) return st;
  }
  const bool down = fused_down(P);
  for (int l = 3; l <= (down ? L - 1 : L); ++l) {
    StageTimer t(P, ST_L2L, s);
    // with the final-stage M2P the leaf locals are the parent's shifted locals
    // alone (the adjoint's P2L wrote them first)
    if ((st = do_l2l(P, tt, l, s, (l == L && P->m2p && !p2l) ? 0 : 1))) return st;
  }
  if (L == 2 && P->m2p && !p2l) {  // no parent far field: the leaf locals are zero
    StageTimer t(P, ST_L2L, s);
    CUDA_TRY(launch_zero<T>(static_cast<T*>(P->Lx(L)), P->lev[L].bytes / sizeof(T), s));
  }
  if (accel && P->near_comps == 4) {  // analytic acceleration, read off the expansions
    StageTimer t(P, ST_LEAF, s);
    CUDA_TRY(launch_leaf_finish_grad<T>(tt, P->lev[L], static_cast<const T*>(P->Lx(L)), near_box,
                                        (P->m2p && !p2l) ? reinterpret_cast<const T*>(P->arena + P->m2p_off) : nullptr,
                                        P->dims, P->G * P->dx * P->dx, -P->G * P->dx, phi, accel, s));
    return FMM_OK;
  }
  {
    StageTimer t(P, ST_LEAF, s);
    LeafDownArgs<T> da;
    if (down) {  // do_l2l's arguments for the leaf level
      da.par = P->lev[L - 1];
      da.Lp = static_cast<const T*>(P->Lx(L - 1));
      da.harm = harmonic_m2l_level(P, L) ? 1 : 0;
      da.Lred = da.harm && P->lev[L].lred_off ? reinterpret_cast<const T*>(P->arena + P->lev[L].lred_off) : nullptr;
    }
    CUDA_TRY(launch_leaf_finish<T>(tt, P->lev[L], static_cast<const T*>(P->Lx(L)), adj_g ? rho_box : near_box,
                                   P->b * P->b * P->b * (adj_g ? 1 : P->near_comps),
                                   (P->m2p && !p2l) ? reinterpret_cast<const T*>(P->arena + P->m2p_off) : nullptr,
                                   P->dims,
                                   P->G * P->dx * P->dx, phi, s, down ? &da : nullptr));
  }
  if (accel) {
    StageTimer t(P, ST_FD, s);
    CUDA_TRY(launch_fd_accel<T>(phi, P->dims, 1.0 / P->dx, accel, s));
  }
  return FMM_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// A host-solve staging buffer, allocated on first use (a failed allocation
// leaves it NULL for the next call to retry).
bool stage_alloc(void** buf, size_t n) {
  if (*buf) return true;
  void* q = nullptr;
  if (cudaMalloc(&q, n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *buf = q;
  return true;
}

}  // namespace

extern "C" {

fmm_status fmm_solve(fmm_plan_t P, const void* rho, void* phi, void* accel, void* stream) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (!rho || !phi) return fail(FMM_ERR_ARG, "rho and phi must be non-NULL");
  if (!aligned16(rho) || !aligned16(phi) || (accel && !aligned16(accel)))
    return fail(FMM_ERR_ARG, "device pointers must be 16-byte aligned");
  if (accel && !P->opts.accel) return fail(FMM_ERR_ARG, "plan was built with accel = 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  P->last_stream = s;
  if (P->f64_data())
    return run_solve<double>(P, static_cast<const double*>(rho), static_cast<double*>(phi),
                             static_cast<double*>(accel), s);
  return run_solve<float>(P, static_cast<const float*>(rho), static_cast<float*>(phi), static_cast<float*>(accel), s);
}

fmm_status fmm_solve_adjoint(fmm_plan_t P, const void* grad_phi, const void* grad_accel, void* grad_rho, void* stream) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (!grad_rho || (!grad_phi && !grad_accel)) return fail(FMM_ERR_ARG, "grad_rho and one gradient must be non-NULL");
  if (grad_accel && !aligned16(grad_accel)) return fail(FMM_ERR_ARG, "device pointers must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  P->last_stream = s;
  void* w = P->arena + P->work_off;
  // the analytic force's transpose runs inside the solve (run_solve); the
  // stencil force's joins the source w through FD^T here
  const bool analytic = grad_accel && P->near_comps == 4;
  const void* fd_g = analytic ? nullptr : grad_accel;
  {
    StageTimer st(P, ST_ADJ_SRC, s);
    if (P->f64_data()) {
      CUDA_TRY(launch_adjoint_source<double>(static_cast<const double*>(grad_phi), static_cast<const double*>(fd_g),
                                             P->dims, 1.0 / P->dx, static_cast<double*>(w), s));
    } else {
      CUDA_TRY(launch_adjoint_source<float>(static_cast<const float*>(grad_phi), static_cast<const float*>(fd_g),
                                            P->dims, 1.0 / P->dx, static_cast<float*>(w), s));
    }
  }
  // mult_order < order: the transpose runs the M2L with the orders swapped
  P->transposed = true;
  P->adj_g = analytic ? grad_accel : nullptr;
  const fmm_status r =
      P->f64_data()
          ? run_solve<double>(P, static_cast<const double*>(w), static_cast<double*>(grad_rho), nullptr, s, true)
          : run_solve<float>(P, static_cast<const float*>(w), static_cast<float*>(grad_rho), nullptr, s, true);
  P->transposed = false;
  P->adj_g = nullptr;
  return r;
}

fmm_status fmm_solve_host(fmm_plan_t P, const void* rho_host, void* phi_host, void* accel_host, void* stream) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (!rho_host || !phi_host) return fail(FMM_ERR_ARG, "rho and phi must be non-NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)P->ncell() * P->esize();
  if (!stage_alloc(&P->d_io_rho, bytes) || !stage_alloc(&P->d_io_phi, bytes) ||
      (accel_host && !stage_alloc(&P->d_io_acc, 3 * bytes)))
    return fail(FMM_ERR_ALLOC, "staging allocation failed");
  CUDA_TRY(cudaMemcpyAsync(P->d_io_rho, rho_host, bytes, cudaMemcpyHostToDevice, s));
  fmm_status st = fmm_solve(P, P->d_io_rho, P->d_io_phi, accel_host ? P->d_io_acc : nullptr, stream);
  if (st != FMM_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(phi_host, P->d_io_phi, bytes, cudaMemcpyDeviceToHost, s));
  if (accel_host) CUDA_TRY(cudaMemcpyAsync(accel_host, P->d_io_acc, 3 * bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return FMM_OK;
}

// Several independent densities through one plan with host buffers: two
// staging sets, the uploads on one copy stream and the downloads on another,
// so that field i + 1's upload and field i's download run beside field i + 1's
// solve.  Set b = i % 2 serves field i; its hazards are waited on explicitly:
// the upload of field i waits for the solve of field i - 2 (which read the
// same rho staging), the solve of field i for that upload and for the
// download of field i - 2 (which read the same phi / accel staging), the
// download of field i for its solve.
fmm_status fmm_solve_host_many(fmm_plan_t P, int count, const void* const* rho_host, void* const* phi_host,
                               void* const* accel_host, void* stream) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (count < 0) return fail(FMM_ERR_ARG, "count %d is negative", count);
  if (count == 0) return FMM_OK;
  if (!rho_host || !phi_host) return fail(FMM_ERR_ARG, "the rho and phi pointer arrays must be non-NULL");
  for (int i = 0; i < count; ++i)
    if (!rho_host[i] || !phi_host[i] || (accel_host && !accel_host[i]))
      return fail(FMM_ERR_ARG, "host buffer of field %d is NULL", i);
  const bool acc = accel_host != nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)P->ncell() * P->esize();
  const bool two = count > 1;
  if (!stage_alloc(&P->d_io_rho, bytes) || !stage_alloc(&P->d_io_phi, bytes) ||
      (acc && !stage_alloc(&P->d_io_acc, 3 * bytes)) ||
      (two && (!stage_alloc(&P->d_io_rho1, bytes) || !stage_alloc(&P->d_io_phi1, bytes) ||
               (acc && !stage_alloc(&P->d_io_acc1, 3 * bytes)))))
    return fail(FMM_ERR_ALLOC, "staging allocation failed");
  if (!P->io_ev[6]) {  // created together, the start event last
    bool ok = cudaStreamCreateWithFlags(&P->io_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&P->io_out, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t& e : P->io_ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {  // none kept: the next call starts over
      cudaGetLastError();
      for (cudaEvent_t& e : P->io_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
      }
      if (P->io_in) cudaStreamDestroy(P->io_in);
      if (P->io_out) cudaStreamDestroy(P->io_out);
      P->io_in = P->io_out = nullptr;
      return fail(FMM_ERR_CUDA, "copy stream or event creation failed");
    }
  }
  void* const R[2] = {P->d_io_rho, P->d_io_rho1};
  void* const F[2] = {P->d_io_phi, P->d_io_phi1};
  void* const A[2] = {P->d_io_acc, P->d_io_acc1};
  cudaEvent_t* const ev = P->io_ev;
  fmm_status st = FMM_OK;
  cudaError_t ce = cudaEventRecord(ev[6], s);  // the copies start after the work queued on `stream`
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(P->io_in, ev[6], 0);
  if (ce == cudaSuccess) ce = cudaStreamWaitEvent(P->io_out, ev[6], 0);
  for (int i = 0; i < count && ce == cudaSuccess; ++i) {
    const int b = i & 1;
    if (i >= 2) ce = cudaStreamWaitEvent(P->io_in, ev[2 + b], 0);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(R[b], rho_host[i], bytes, cudaMemcpyHostToDevice, P->io_in);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[b], P->io_in);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ev[b], 0);
    if (ce == cudaSuccess && i >= 2) ce = cudaStreamWaitEvent(s, ev[4 + b], 0);
    if (ce != cudaSuccess) break;
    st = fmm_solve(P, R[b], F[b], acc ? A[b] : nullptr, stream);
    if (st != FMM_OK) break;
    ce = cudaEventRecord(ev[2 + b], s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(P->io_out, ev[2 + b], 0);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(phi_host[i], F[b], bytes, cudaMemcpyDeviceToHost, P->io_out);
    if (ce == cudaSuccess && acc)
      ce = cudaMemcpyAsync(accel_host[i], A[b], 3 * bytes, cudaMemcpyDeviceToHost, P->io_out);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[4 + b], P->io_out);
  }
  // every copy drained before returning, after an error too
  const cudaError_t e1 = cudaStreamSynchronize(P->io_in);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  const cudaError_t e3 = cudaStreamSynchronize(P->io_out);
  if (st != FMM_OK) return st;
  if (ce == cudaSuccess) ce = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
  if (ce != cudaSuccess) return fail(FMM_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(ce));
  return FMM_OK;
}

fmm_status fmm_check(fmm_plan_t P) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  CUDA_TRY(cudaStreamSynchronize(P->last_stream));
  int flag = 0;
  CUDA_TRY(cudaMemcpy(&flag, P->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CUDA_TRY(cudaMemset(P->d_flag, 0, sizeof(int)));
    if (flag & 1)
      return fail(FMM_ERR_NONFINITE, "the density held a NaN or Inf%s",
                  (flag & 2) ? " (and a device wait reached its time limit)" : "");
    return fail(FMM_ERR_TIMEOUT, "a device wait reached its time limit (wait sites 0x%x)", (flag >> 8) & 0xff);
  }
  return FMM_OK;
}

size_t fmm_workspace_bytes(fmm_plan_t P) { return P ? P->dev_bytes : 0; }

int fmm_plan_leaf_level(fmm_plan_t P) { return P ? P->L : -1; }

int fmm_plan_level_kind(fmm_plan_t P, int level) {
  if (!P || level < 0 || level > P->L) return -1;
  if (level < 2) return 0;
  const Level& lv = P->lev[level];
  return lv.tc ? 3 : (lv.f64 ? 2 : 1);
}

int fmm_plan_near_on_tensor_cores(fmm_plan_t P) { return (P && P->near_tc) ? 1 : 0; }

int fmm_solve_launches(fmm_plan_t P, int with_accel) {
  if (!P) return -1;
  const int L = P->L;
  int n = 1;                            // P2M (with the finite check)
  n += std::max(0, L - 2);              // M2M for l = L .. 3
  if (fused_down(P)) n -= 1;            // the last L2L inside the leaf kernel
  if (L < 2) n += 1;                    // zero the leaf locals
  for (int l = 2; l <= L; ++l) {
    n += l >= 3 ? 2 : 1;                // M2L, and L2L below level 2
    if (l == 2 && harmonic_m2l_level(P, 2)) n += 1;  // rebuild of the harmonic level-2 locals
    if (l == 2 && L == 2 && P->m2p) n += 1;          // zero leaf locals (final-stage M2P, no parent far field)
    if (!P->lev[l].tc && P->m2l_choice[l].dsplit > 1 && !(l == L && P->m2p)) n += 1;  // partial-sum reduction
  }
  n += P->near_tc ? ((P->near4 && P->use_near4) || tc_prefix(P, TS_NEAR) ? 1 : (int)P->tcn.size()) + 1
                   : 2;  // near field + leaf finish
  if (!P->near_tc && P->near_choice.dsplit > 1) n += 1;
  if (with_accel && P->near_comps == 1) n += 1;  // FD stencil (the analytic force comes with the leaf kernel)
  return n;
}

fmm_status fmm_timing_enable(fmm_plan_t P, int enable) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (enable && P->ev_pool.empty()) {  // the whole pool or none of it
    std::vector<cudaEvent_t> pool;
    pool.reserve(kEventPool);
    for (int i = 0; i < kEventPool; ++i) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        for (cudaEvent_t f : pool) cudaEventDestroy(f);
        return fail(FMM_ERR_CUDA, "timing event creation failed");
      }
      pool.push_back(e);
    }
    P->ev_pool = std::move(pool);
  }
  CUDA_TRY(cudaDeviceSynchronize());
  P->recs.clear();
  P->ev_used = 0;
  P->timing = enable != 0;
  return FMM_OK;
}

fmm_status fmm_timing_read(fmm_plan_t P, double* ms, int* launches, int nstages) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (!ms || !launches || nstages <= 0) return fail(FMM_ERR_ARG, "bad output arrays");
  CUDA_TRY(cudaDeviceSynchronize());
  for (int i = 0; i < nstages; ++i) ms[i] = 0.0, launches[i] = 0;
  for (const auto& r : P->recs) {
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    if (r.stage < nstages) {
      ms[r.stage] += t;
      launches[r.stage] += 1;
    }
  }
  P->recs.clear();
  P->ev_used = 0;
  return FMM_OK;
}

int fmm_timing_stage_count(void) { return ST_COUNT; }

const char* fmm_timing_stage_name(int stage) {
  return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}

fmm_status fmm_plan_destroy(fmm_plan_t P) {
  if (!P) return FMM_OK;
  P->release();
  delete P;
  return FMM_OK;
}

fmm_status fmm_debug_level(fmm_plan_t P, int what, int level, double* host_out, size_t host_count) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (what != 0 && what != 1) return fail(FMM_ERR_ARG, "what must be 0 or 1");
  if (level < P->lmin || level > P->L) return fail(FMM_ERR_ARG, "level %d not stored", level);
  const Level& lv = P->lev[level];
  const size_t count = (size_t)lv.nbox * P->nc;
  if (!host_out || host_count < count) return fail(FMM_ERR_ARG, "host buffer too small (%zu needed)", count);
  double* tmp = nullptr;
  CUDA_TRY(cudaMalloc(&tmp, count * sizeof(double)));
  const double h = (double)P->b * (double)(1LL << (P->L - level));
  const void* src = what == 0 ? P->M(level) : P->Lx(level);
  void* full = nullptr;  // leaf locals with the fused last L2L: that L2L, into a copy of the M2L's locals
  if (what == 1 && level == P->L && fused_down(P)) {
    cudaError_t e = cudaMalloc(&full, lv.bytes);
    if (e == cudaSuccess) e = cudaMemcpy(full, P->Lx(level), lv.bytes, cudaMemcpyDeviceToDevice);
    const Level& q = P->lev[level - 1];
    const int harm = harmonic_m2l_level(P, level) ? 1 : 0;
    const void* red = harm && lv.lred_off ? P->arena + lv.lred_off : nullptr;
    if (e == cudaSuccess)
      e = lv.f64 ? launch_l2l<double, double>(P->tables(), q, static_cast<const double*>(P->Lx(level - 1)), lv,
                                              static_cast<double*>(full), 1, harm, static_cast<const double*>(red), 0)
                 : launch_l2l<float, float>(P->tables(), q, static_cast<const float*>(P->Lx(level - 1)), lv,
                                            static_cast<float*>(full), 1, harm, static_cast<const float*>(red), 0);
    if (e != cudaSuccess) {
      if (full) cudaFree(full);
      cudaFree(tmp);
      return fail(FMM_ERR_CUDA, "debug export failed: %s", cudaGetErrorString(e));
    }
    src = full;
  }
  cudaError_t e = lv.f64 ? launch_export_level<double>(static_cast<const double*>(src), lv, what, h, P->d_mi, P->nc,
                                                       tmp, nullptr)
                         : launch_export_level<float>(static_cast<const float*>(src), lv, what, h, P->d_mi, P->nc, tmp,
                                                      nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host_out, tmp, count * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (full) cudaFree(full);
  if (e != cudaSuccess) return fail(FMM_ERR_CUDA, "debug export failed: %s", cudaGetErrorString(e));
  return FMM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve: the workspace is a file-scope static device array.
namespace {

constexpr size_t kStaticWorkspaceBytes = FMM_STATIC_WORKSPACE_BYTES;
constexpr int kStaticMaxOrder = 6;
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

// Per device: the array's device address (looked up on every call, with the
// device current: a device reset gives the array a new address, whose
// contents are then not the tables of the last call) and the (order, leaf,
// nx, ny, nz) whose tables the array holds.
struct StaticSlot {
  unsigned char* ptr = nullptr;
  int key[5] = {-1, -1, -1, -1, -1};
};
StaticSlot g_static_slots[kStaticMaxDevices];
std::mutex g_static_mutex;

}  // namespace

extern "C" fmm_status fmm_solve_static(const fmm_grid* grid, int order, int leaf, const void* rho, void* phi,
                                       void* accel, void* stream) {
  g_last_error.clear();
  if (!grid) return fail(FMM_ERR_ARG, "grid is NULL");
  if (order < 0 || order > kStaticMaxOrder)
    return fail(FMM_ERR_ARG, "order %d outside [0, %d] for the static workspace", order, kStaticMaxOrder);
  if (leaf != 2 && leaf != 4 && leaf != 8) return fail(FMM_ERR_ARG, "leaf %d not in {2, 4, 8}", leaf);
  const int d3[3] = {grid->nx, grid->ny, grid->nz};
  for (int q = 0; q < 3; ++q) {
    if (d3[q] <= 0) return fail(FMM_ERR_ARG, "grid extent %d must be positive", d3[q]);
    if (d3[q] % leaf) return fail(FMM_ERR_ARG, "grid extent %d is not a multiple of leaf %d", d3[q], leaf);
    if (d3[q] > 4096) return fail(FMM_ERR_ARG, "grid extent %d too large for the static workspace", d3[q]);
  }
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx)) return fail(FMM_ERR_ARG, "dx must be positive and finite");
  if (!std::isfinite(grid->G)) return fail(FMM_ERR_ARG, "G must be finite");
  if (!rho || !phi) return fail(FMM_ERR_ARG, "rho and phi must be non-NULL");
  if (!aligned16(rho) || !aligned16(phi) || (accel && !aligned16(accel)))
    return fail(FMM_ERR_ARG, "device pointers must be 16-byte aligned");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(FMM_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticSlot& slot = g_static_slots[dev];
  {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_workspace);
    if (e != cudaSuccess || !addr)
      return fail(FMM_ERR_CUDA, "cudaGetSymbolAddress of the static workspace failed: %s", cudaGetErrorString(e));
    if (static_cast<unsigned char*>(addr) != slot.ptr) {  // first call, or a new context: no tables held
      slot.ptr = static_cast<unsigned char*>(addr);
      for (int& k : slot.key) k = -1;
    }
  }
  std::unique_ptr<fmm_plan_s> P(new (std::nothrow) fmm_plan_s());
  if (!P) return fail(FMM_ERR_ALLOC, "host allocation failed");
  P->static_base = slot.ptr;
  P->static_cap = kStaticWorkspaceBytes;
  P->no_split = true;  // no neighbour-split scratch
  const int key[5] = {order, leaf, d3[0], d3[1], d3[2]};
  P->static_keep_tables = std::equal(key, key + 5, slot.key);
  fmm_opts o;
  fmm_default_opts(&o);  // FP32 on the CUDA cores
  o.m2l_cartesian = 1;     // no folded arrays: the workspace limit stays that of the plain contraction
  fmm_status st = plan_init(P.get(), d3, grid->dx, grid->G, order, leaf, o, s, dev);
  if (st != FMM_OK) {
    for (int& k : slot.key) k = -1;  // the tables may be half written
    return st;
  }
  std::copy(key, key + 5, slot.key);
  // plan_init cleared the arena; the flag word is kept with the tables
  CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), s));
  st = run_solve<float>(P.get(), static_cast<const float*>(rho), static_cast<float*>(phi),
                        static_cast<float*>(accel), s);
  // nothing of P was allocated on the device: no release
  return st;
}

// ---------------------------------------------------------------------------
// Batched solves under one CUDA graph.
// One launch of a fused batch: a multi-item kernel over the items whose
// arguments and grids sit in the batch's device table.
namespace {
enum MultiKind { MK_P2M, MK_M2M, MK_GEMM, MK_L2L, MK_LEAF, MK_FD };
struct MultiStep {
  int kind = 0, shape = 0, n = 0, bs = 0, harm_rows = 0;
  long long blocks = 0;
  size_t args_off = 0, grids_off = 0;
};
}  // namespace

struct fmm_batch_s {
  std::vector<fmm_plan_t> plans;
  std::vector<cudaStream_t> side;  // one capture branch per plan (reused round-robin)
  std::vector<cudaEvent_t> ev;     // fork / join events
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;    // buffers the graph was captured with
  bool with_accel = false;
  // Fused form: each step kind one launch over every field (multi.cuh)
  bool allow_fused = true;
  int fused = -1;                  // the graph holds: -1 nothing yet, 0 per-field solves, 1 fused steps
  std::vector<MultiStep> steps;
  std::vector<unsigned char> h_tab;  // item arguments and grids, as uploaded
  unsigned char* d_tab = nullptr;
  size_t d_tab_cap = 0;
  // the contraction launches of the fused form run side by side: streams
  // and fork / join events
  cudaStream_t fk[5] = {};  // one per contraction shape after the first
  cudaEvent_t fev[6] = {};
};

namespace {
void batch_free_graph(fmm_batch_t B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

// Whether the plans of a batch run fused: CUDA-core plans (no tensor-core
// level, near field or final-stage M2P) of one order whose levels all hold
// the data's precision, with the stencil force where a force is asked for
// (the FP32 stencil kernel; FP64 forces keep the per-field graph).
bool batch_fusable_plans(fmm_batch_t B, bool with_accel) {
  const fmm_plan_t P0 = B->plans[0];
  for (fmm_plan_t P : B->plans) {
    if (P->p != P0->p || P->f64_data() != P0->f64_data() || P->L < 2 || P->near_tc || P->m2p) return false;
    for (int l = 2; l <= P->L; ++l)
      if (P->lev[l].tc || P->lev[l].f64 != P->f64_data()) return false;
    if (with_accel && (!P->opts.accel || P->near_comps != 1 || P->f64_data() || P->dims[0] % 4 != 0)) return false;
  }
  return true;
}

template <typename A>
size_t tab_put(std::vector<unsigned char>& tab, const A* v, size_t n) {
  const size_t off = (tab.size() + 15) & ~(size_t)15;
  tab.resize(off + n * sizeof(A));
  if (n) std::memcpy(tab.data() + off, v, n * sizeof(A));
  return off;
}

// Appends one step of items (those with no blocks left out).
template <typename A>
void add_step(fmm_batch_t B, int kind, int shape, int bs, int harm_rows, const std::vector<A>& args,
              const std::vector<std::array<unsigned, 3>>& grids) {
  std::vector<A> a;
  std::vector<MultiGrid> g;
  long long start = 0;
  for (size_t i = 0; i < args.size(); ++i) {
    const long long nb = (long long)grids[i][0] * grids[i][1] * grids[i][2];
    if (nb <= 0) continue;
    a.push_back(args[i]);
    MultiGrid m{};
    m.gx = grids[i][0];
    m.gy = grids[i][1];
    m.gz = grids[i][2];
    m.start = start;
    g.push_back(m);
    start += nb;
  }
  if (a.empty()) return;
  MultiStep st;
  st.kind = kind;
  st.shape = shape;
  st.bs = bs;
  st.harm_rows = harm_rows;
  st.n = (int)a.size();
  st.blocks = start;
  st.args_off = tab_put(B->h_tab, a.data(), a.size());
  st.grids_off = tab_put(B->h_tab, g.data(), g.size());
  B->steps.push_back(st);
}

// Tile shape of a contraction inside the fused batch, where the other
// fields fill the GPU: the z-run tiles of the longer run (the fastest per
// row); a grid of at most 64 rows takes the tiny-grid form (shape 4: real
// rows and in-grid neighbours only; the 4 x 4 x 4 tile took 3 ms of the
// 64-field step on them, the column-per-lane form longer).
int batch_shape(const NbrGemm& g, const std::vector<int>& tile_k, bool fp32) {
  if (nbr_gemm_tiny_fits(g)) return 4;
  if (!zrun_eligible(g, tile_k.data(), g.ntiles)) return g.shape;
  // FP32: RZ = 8, or RZ = 6 (shape 5) where it pads the z extent less (12^3
  // and 6^3 rows: RZ = 8 pads them to 16 and 8); RZ = 4 pads like RZ = 6 at
  // a lower rate per row (on the 12^3 grids it measured the same as RZ = 8)
  const int z = g.grid[2];
  return fp32 && (z + 5) / 6 * 6 < (z + 7) / 8 * 8 ? 5 : 1;
}

std::array<unsigned, 3> blocks_1d(long long threads, int bs) {
  return {(unsigned)((threads + bs - 1) / bs), 1u, 1u};
}

// The fused schedule (Sec. 2.3's steps, each over every field): P2M; M2M by
// depth below the leaf level; every field's M2L levels and near field
// together, one launch per contraction shape; L2L by absolute level (the
// level-2 harmonic rebuild first); the leaf evaluation; the stencil force.
// Buffers may be NULL when only the step count is wanted.
template <typename T>
void build_fused(fmm_batch_t B, const void* const* rho, void* const* phi, void* const* accel, bool with_accel) {
  B->steps.clear();
  B->h_tab.clear();
  const int n = (int)B->plans.size();
  constexpr int bs = 256;  // block size of the tree kernels (M2M, L2L)
  int maxL = 0;
  for (fmm_plan_t P : B->plans) maxL = std::max(maxL, P->L);
  {  // P2M (and the near field's box-major density)
    std::vector<P2mArgs> a;
    std::vector<std::array<unsigned, 3>> g;
    int harm_rows = 0;
    for (int i = 0; i < n; ++i) {
      const fmm_plan_t P = B->plans[i];
      const Level& lf = P->lev[P->L];
      P2mArgs x{};
      x.rho = rho ? rho[i] : nullptr;
      x.nx = P->dims[0];
      x.ny = P->dims[1];
      x.b = P->b;
      x.leaf = lf;
      x.Mleaf = P->M(P->L);
      x.rho_box = P->arena + P->rho_box_off;
      x.flag = P->d_flag;
      x.harm = lf.fold_off ? 1 : 0;
      x.Mfold = lf.fold_off ? P->arena + lf.fold_off : nullptr;
      x.ncell = P->ncell();
      harm_rows |= x.harm;
      a.push_back(x);
      g.push_back(blocks_1d(lf.npar * 16, 256));
    }
    add_step(B, MK_P2M, 0, 256, harm_rows, a, g);
  }
  for (int k = 0; k + 3 <= maxL; ++k) {  // M2M: level L - k to L - k - 1 of every field deep enough
    std::vector<M2mArgs> a;
    std::vector<std::array<unsigned, 3>> g;
    for (fmm_plan_t P : B->plans) {
      const int l = P->L - k;
      if (l < 3) continue;
      const Level &c = P->lev[l], &q = P->lev[l - 1];
      M2mArgs x{};
      x.child = c;
      x.Mc = P->M(l);
      x.par = q;
      x.Mp = P->M(l - 1);
      x.harm = q.fold_off ? 1 : 0;
      x.Mfold = q.fold_off ? P->arena + q.fold_off : nullptr;
      a.push_back(x);
      g.push_back(blocks_1d(c.npar * 8, bs));
    }
    add_step(B, MK_M2M, 0, bs, 0, a, g);
  }
  {  // M2L of every level and the near field: independent contractions
    std::vector<NbrGemm> a[6];
    std::vector<std::array<unsigned, 3>> g[6];
    auto add = [&](NbrGemm x, const std::vector<int>& tile_k) {
      x.dsplit = 1;  // the batch fills the GPU: no neighbour split, no partial sums
      x.partial = nullptr;
      x.max_blocks = 0;
      x.shape = batch_shape(x, tile_k, sizeof(T) == 4);
      std::array<unsigned, 3> gr;
      if (x.shape == 4)
        gr = {(unsigned)x.ntiles, 1u, 1u};
      else if (x.shape == 5)
        nbr_gemm_zrun_grid<T>(x, 2, gr.data());
      else if (x.shape == 1 || x.shape == 2)
        nbr_gemm_zrun_grid<T>(x, x.shape - 1, gr.data());
      else
        nbr_gemm_simt_col_grid<T>(x, gr.data());
      a[x.shape].push_back(x);
      g[x.shape].push_back(gr);
    };
    for (fmm_plan_t P : B->plans) {
      for (int l = 2; l <= P->L; ++l) add(m2l_gemm(P, l), P->h_m2l_tile_k);
      add(near_gemm(P), P->h_near_tile_k);
    }
    for (int sh : {1, 5, 0, 2, 3, 4}) add_step(B, MK_GEMM, sh, 0, 0, a[sh], g[sh]);  // the tiny-grid launch last
  }
  for (int l = 2; l <= maxL; ++l) {  // L2L, coarse to fine (a fused leaf level's in the leaf kernel)
    std::vector<L2lArgs> a;
    std::vector<std::array<unsigned, 3>> g;
    for (fmm_plan_t P : B->plans) {
      if (l > P->L || (l == P->L && fused_down(P))) continue;
      const bool harm = harmonic_m2l_level(P, l);
      if (l == 2 && !harm) continue;  // level-2 locals are its M2L alone
      const Level &q = P->lev[l - 1], &c = P->lev[l];
      L2lArgs x{};
      x.par = q;
      x.Lp = l == 2 ? nullptr : P->Lx(l - 1);
      x.child = c;
      x.Lc = P->Lx(l);
      x.accumulate = 1;
      x.harm = harm ? 1 : 0;
      x.Lred = harm && c.lred_off ? P->arena + c.lred_off : nullptr;
      a.push_back(x);
      g.push_back(blocks_1d(q.nbox * 8, bs));
    }
    add_step(B, MK_L2L, 0, bs, 0, a, g);
  }
  {  // leaf evaluation: L2P plus the near field, scaled
    std::vector<LeafArgs> a;
    std::vector<std::array<unsigned, 3>> g;
    for (int i = 0; i < n; ++i) {
      const fmm_plan_t P = B->plans[i];
      LeafArgs x{};
      x.leaf = P->lev[P->L];
      x.Lleaf = P->Lx(P->L);
      x.near_box = P->arena + P->near_off;
      x.near_stride = P->b * P->b * P->b * P->near_comps;
      x.nx = P->dims[0];
      x.ny = P->dims[1];
      x.b = P->b;
      x.scale = P->G * P->dx * P->dx;
      x.phi = phi ? phi[i] : nullptr;
      if (fused_down(P)) {  // run_solve's arguments for the leaf level's L2L
        const int L = P->L;
        x.par = P->lev[L - 1];
        x.Lp = P->Lx(L - 1);
        x.harm = harmonic_m2l_level(P, L) ? 1 : 0;
        x.Lred = x.harm && P->lev[L].lred_off ? P->arena + P->lev[L].lred_off : nullptr;
      }
      a.push_back(x);
      g.push_back(blocks_1d(x.leaf.npar * 8, 256));
    }
    add_step(B, MK_LEAF, 0, 256, 0, a, g);
  }
  if (with_accel) {  // force by the 5-point stencil (App. C)
    std::vector<FdArgs> a;
    std::vector<std::array<unsigned, 3>> g;
    for (int i = 0; i < n; ++i) {
      const fmm_plan_t P = B->plans[i];
      FdArgs x{};
      x.phi = phi ? phi[i] : nullptr;
      x.nx = P->dims[0];
      x.ny = P->dims[1];
      x.nz = P->dims[2];
      x.inv_dx = 1.0 / P->dx;
      x.accel = accel ? accel[i] : nullptr;
      std::array<unsigned, 3> gr;
      fd_multi_grid(P->dims, gr.data());
      a.push_back(x);
      g.push_back(gr);
    }
    add_step(B, MK_FD, 0, 0, 0, a, g);
  }
}

// The steps in order, except that the contraction launches (independent of
// one another) run side by side: the first on `s`, the others on the fork
// streams, joined before the next step.  The z-run launch goes first and
// the tiny-grid launch (few latency-bound blocks) last: its blocks then take
// the SMs the z-run blocks free (27.9 -> 27.7 ms for the 64-field batch,
// against starting them first).
template <typename T>
fmm_status run_fused(fmm_batch_t B, cudaStream_t s) {
  const int p = B->plans[0]->p;
  int ngemm = 0, nfork = 0;
  for (const MultiStep& st : B->steps) ngemm += st.kind == MK_GEMM;
  for (const MultiStep& st : B->steps) {
    const void* a = B->d_tab + st.args_off;
    const MultiGrid* g = reinterpret_cast<const MultiGrid*>(B->d_tab + st.grids_off);
    cudaError_t e = cudaSuccess;
    cudaStream_t ls = s;
    if (st.kind == MK_GEMM && ngemm > 1) {
      if (nfork == 0) CUDA_TRY(cudaEventRecord(B->fev[0], s));
      if (nfork > 0) {  // the fork streams (at most five more contraction shapes)
        ls = B->fk[nfork - 1];
        CUDA_TRY(cudaStreamWaitEvent(ls, B->fev[0], 0));
      }
      ++nfork;
    }
    if (st.kind != MK_GEMM && nfork > 1) {  // join the fork streams
      for (int k = 1; k < nfork; ++k) {
        CUDA_TRY(cudaEventRecord(B->fev[k], B->fk[k - 1]));
        CUDA_TRY(cudaStreamWaitEvent(s, B->fev[k], 0));
      }
      nfork = 0;
      ngemm = 0;
    }
    switch (st.kind) {
      case MK_P2M:
        e = launch_p2m_multi<T>(p, static_cast<const P2mArgs*>(a), g, st.n, st.blocks, st.harm_rows, ls);
        break;
      case MK_M2M:
        e = launch_m2m_multi<T, T>(p, static_cast<const M2mArgs*>(a), g, st.n, st.blocks, st.bs, ls);
        break;
      case MK_GEMM: {
        const NbrGemm* gs = static_cast<const NbrGemm*>(a);
        if (st.shape == 4)
          e = launch_nbr_gemm_tiny_multi<T>(gs, g, st.n, st.blocks, ls);
        else if (st.shape == 0)
          e = launch_nbr_gemm_simt_multi<T>(gs, g, st.n, st.blocks, ls);
        else if (st.shape == 3)
          e = launch_nbr_gemm_col_multi<T>(gs, g, st.n, st.blocks, ls);
        else if (st.shape == 5)
          e = launch_nbr_gemm_zrun_multi<T>(2, gs, g, st.n, st.blocks, ls);
        else
          e = launch_nbr_gemm_zrun_multi<T>(st.shape - 1, gs, g, st.n, st.blocks, ls);
        break;
      }
      case MK_L2L:
        e = launch_l2l_multi<T, T>(p, static_cast<const L2lArgs*>(a), g, st.n, st.blocks, st.bs, ls);
        break;
      case MK_LEAF:
        e = launch_leaf_finish_multi<T>(p, static_cast<const LeafArgs*>(a), g, st.n, st.blocks, ls);
        break;
      case MK_FD:
        e = launch_fd_accel_multi(static_cast<const FdArgs*>(a), g, st.n, st.blocks, ls);
        break;
    }
    CUDA_TRY(e);
  }
  return FMM_OK;
}

// Builds the fused schedule for these buffers and uploads its table.
fmm_status prepare_fused(fmm_batch_t B, const void* const* rho, void* const* phi, void* const* accel) {
  if (B->plans[0]->f64_data())
    build_fused<double>(B, rho, phi, accel, accel != nullptr);
  else
    build_fused<float>(B, rho, phi, accel, accel != nullptr);
  const size_t bytes = std::max<size_t>(B->h_tab.size(), 16);
  // a graph launched on any stream may still read the previous table
  CUDA_TRY(cudaDeviceSynchronize());
  if (bytes > B->d_tab_cap) {
    if (B->d_tab) cudaFree(B->d_tab);
    B->d_tab = nullptr;
    B->d_tab_cap = 0;
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(FMM_ERR_ALLOC, "cudaMalloc(%zu) of the batch table failed", bytes);
    }
    B->d_tab = static_cast<unsigned char*>(d);
    B->d_tab_cap = bytes;
  }
  CUDA_TRY(cudaMemcpy(B->d_tab, B->h_tab.data(), B->h_tab.size(), cudaMemcpyHostToDevice));
  return FMM_OK;
}

fmm_status run_fused_any(fmm_batch_t B, cudaStream_t s) {
  return B->plans[0]->f64_data() ? run_fused<double>(B, s) : run_fused<float>(B, s);
}
}  // namespace

extern "C" fmm_status fmm_batch_create(const fmm_plan_t* plans, int count, fmm_batch_t* out) {
  g_last_error.clear();
  if (!out) return fail(FMM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!plans || count <= 0) return fail(FMM_ERR_ARG, "need at least one plan");
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return fail(FMM_ERR_ARG, "plan %d is NULL", i);
  fmm_batch_t B = new (std::nothrow) fmm_batch_s();
  if (!B) return fail(FMM_ERR_ALLOC, "host allocation failed");
  B->plans.assign(plans, plans + count);
  const int nside = std::min(count, 32);
  B->side.resize(nside, nullptr);
  for (auto& st : B->side)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      fmm_batch_destroy(B);
      return fail(FMM_ERR_CUDA, "stream creation failed");
    }
  B->ev.resize(nside + 1, nullptr);
  for (auto& e : B->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      fmm_batch_destroy(B);
      return fail(FMM_ERR_CUDA, "event creation failed");
    }
  for (auto& st : B->fk)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      fmm_batch_destroy(B);
      return fail(FMM_ERR_CUDA, "stream creation failed");
    }
  for (auto& e : B->fev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      fmm_batch_destroy(B);
      return fail(FMM_ERR_CUDA, "event creation failed");
    }
  *out = B;
  return FMM_OK;
}

extern "C" fmm_status fmm_batch_solve(fmm_batch_t B, const void* const* rho, void* const* phi, void* const* accel,
                                      void* stream) {
  if (!B) return fail(FMM_ERR_ARG, "batch is NULL");
  if (!rho || !phi) return fail(FMM_ERR_ARG, "rho and phi arrays must be non-NULL");
  const int n = (int)B->plans.size();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void*> key;
  key.reserve(3 * n);
  for (int i = 0; i < n; ++i) {
    if (!rho[i] || !phi[i]) return fail(FMM_ERR_ARG, "rho[%d] / phi[%d] is NULL", i, i);
    key.push_back(rho[i]);
    key.push_back(phi[i]);
    key.push_back(accel ? accel[i] : nullptr);
  }
  if (!B->exec || key != B->key) {
    batch_free_graph(B);
    B->fused = -1;
    bool fuse = B->allow_fused && batch_fusable_plans(B, accel != nullptr);
    for (int i = 0; i < n && fuse; ++i)
      fuse = aligned16(rho[i]) && aligned16(phi[i]) && (!accel || (accel[i] && aligned16(accel[i])));
    if (fuse) {
      fmm_status st = prepare_fused(B, rho, phi, accel);
      if (st != FMM_OK) return st;
      // one eager pass: first-use set-up must not happen inside a capture
      if ((st = run_fused_any(B, s)) != FMM_OK) return st;
      CUDA_TRY(cudaStreamSynchronize(s));
      cudaStream_t cap = B->side[0];
      CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      st = run_fused_any(B, cap);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(cap, &g);
      if (st != FMM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (ec != cudaSuccess) return fail(FMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
      B->graph = g;
      if (cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
        batch_free_graph(B);
        return fail(FMM_ERR_CUDA, "graph instantiation failed");
      }
      B->key = key;
      B->with_accel = accel != nullptr;
      B->fused = 1;
      for (auto* P : B->plans) P->last_stream = s;
      CUDA_TRY(cudaGraphLaunch(B->exec, s));
      return FMM_OK;
    }
    // one eager solve per plan: first-use set-up (kernel attributes, lazy
    // module loading) must not happen inside a capture
    for (int i = 0; i < n; ++i) {
      fmm_plan_t P = B->plans[i];
      const bool timing = P->timing;
      P->timing = false;
      fmm_status st = fmm_solve(P, rho[i], phi[i], accel ? accel[i] : nullptr, stream);
      P->timing = timing;
      if (st != FMM_OK) return st;
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    cudaStream_t cap = B->side[0];
    CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    fmm_status st = FMM_OK;
    const int nside = (int)B->side.size();
    // fork: every side stream waits on the capture origin
    if (cudaEventRecord(B->ev[0], cap) != cudaSuccess) st = fail(FMM_ERR_CUDA, "capture fork failed");
    for (int k = 1; k < nside && st == FMM_OK; ++k)
      if (cudaStreamWaitEvent(B->side[k], B->ev[0], 0) != cudaSuccess) st = fail(FMM_ERR_CUDA, "capture fork failed");
    for (int i = 0; i < n && st == FMM_OK; ++i) {
      fmm_plan_t P = B->plans[i];
      const bool timing = P->timing;
      P->timing = false;
      st = fmm_solve(P, rho[i], phi[i], accel ? accel[i] : nullptr, B->side[i % nside]);
      P->timing = timing;
    }
    // join
    for (int k = 1; k < nside && st == FMM_OK; ++k) {
      if (cudaEventRecord(B->ev[k], B->side[k]) != cudaSuccess ||
          cudaStreamWaitEvent(cap, B->ev[k], 0) != cudaSuccess)
        st = fail(FMM_ERR_CUDA, "capture join failed");
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &g);
    if (st != FMM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ec != cudaSuccess) return fail(FMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
    B->graph = g;
    if (cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
      batch_free_graph(B);
      return fail(FMM_ERR_CUDA, "graph instantiation failed");
    }
    B->key = key;
    B->with_accel = accel != nullptr;
    B->fused = 0;
  }
  for (auto* P : B->plans) P->last_stream = s;  // fmm_check waits on the graph's stream
  CUDA_TRY(cudaGraphLaunch(B->exec, s));
  return FMM_OK;
}

extern "C" fmm_status fmm_batch_destroy(fmm_batch_t B) {
  if (!B) return FMM_OK;
  batch_free_graph(B);
  if (B->d_tab) {
    cudaDeviceSynchronize();  // a launched graph may still read the table
    cudaFree(B->d_tab);
  }
  for (auto& st : B->side)
    if (st) cudaStreamDestroy(st);
  for (auto& e : B->ev)
    if (e) cudaEventDestroy(e);
  for (auto& st : B->fk)
    if (st) cudaStreamDestroy(st);
  for (auto& e : B->fev)
    if (e) cudaEventDestroy(e);
  delete B;
  return FMM_OK;
}

extern "C" int fmm_batch_launches(fmm_batch_t B, int with_accel) {
  if (!B) return -1;
  if (B->allow_fused && batch_fusable_plans(B, with_accel != 0)) {
    // the fused schedule's step count (the buffers do not change it); the
    // table held for the current buffers is left as it is
    std::vector<MultiStep> keep_steps;
    std::vector<unsigned char> keep_tab;
    keep_steps.swap(B->steps);
    keep_tab.swap(B->h_tab);
    if (B->plans[0]->f64_data())
      build_fused<double>(B, nullptr, nullptr, nullptr, with_accel != 0);
    else
      build_fused<float>(B, nullptr, nullptr, nullptr, with_accel != 0);
    const int count = (int)B->steps.size();
    keep_steps.swap(B->steps);
    keep_tab.swap(B->h_tab);
    return count;
  }
  int n = 0;
  for (auto* P : B->plans) n += fmm_solve_launches(P, with_accel);
  return n;
}

extern "C" fmm_status fmm_batch_set_fused(fmm_batch_t B, int enable) {
  if (!B) return fail(FMM_ERR_ARG, "batch is NULL");
  if ((enable != 0) != B->allow_fused) {
    B->allow_fused = enable != 0;
    batch_free_graph(B);
    B->key.clear();
  }
  return FMM_OK;
}

extern "C" int fmm_batch_is_fused(fmm_batch_t B) { return B ? B->fused : -1; }

// ---------------------------------------------------------------------------
// Autotuner of the CUDA-core contractions (M2L levels off the tensor cores and
// the near field): each candidate tile shape / neighbour split is timed on the
// plan's own buffers and the fastest kept.  Results are cached per process by
// contraction geometry, so plans of the same shape tune once.
namespace {

using SimtChoice = fmm_plan_s::SimtChoice;
std::mutex g_tune_mu;
std::map<std::string, SimtChoice> g_tune_cache;
std::map<std::string, int> g_tc_tune_cache;  // tensor-core schedule: 0 span, 1 prefix, 2 dedicated near field

bool choice_valid(fmm_plan_t P, NbrGemm g, const std::vector<int>& tk, size_t es, SimtChoice c) {
  // FP64 levels of a tensor-core plan keep the small-footprint tile that can
  // share an SM with a tensor-core CTA
  if ((c.shape == 1 || c.shape == 2) && es == 8 && P->tc_kind >= 0) return false;
  const size_t one = (size_t)g.grid[0] * g.grid[1] * g.grid[2] * (size_t)g.n_cols * es;
  if (c.dsplit > 1 && (size_t)c.dsplit * one > P->part_cap) return false;
  if (c.shape == 0 || c.shape == 3) return c.dsplit == 1 || c.dsplit == 27;
  if (c.shape != 1 && c.shape != 2) return false;
  g.dsplit = c.dsplit;
  return zrun_eligible(g, tk.data(), (int)tk.size());
}

template <typename T>
fmm_status tune_one(fmm_plan_t P, NbrGemm g, const std::vector<int>& tk, const char* what, int reps, cudaStream_t s,
                    SimtChoice* out) {
  char key[160];
  std::snprintf(key, sizeof key, "%s/%zu/%d,%d,%d/%d/%d/%d/%d/%d", what, sizeof(T), g.grid[0], g.grid[1], g.grid[2],
                g.row_len, g.n_cols, g.ntiles, P->p, P->b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && choice_valid(P, g, tk, sizeof(T), it->second)) {
      *out = it->second;
      return FMM_OK;
    }
  }
  std::vector<SimtChoice> cand;
  const SimtChoice all[] = {{0, 1}, {0, 27}, {1, 1}, {1, 3}, {1, 9}, {2, 1}, {2, 3}, {2, 9}, {3, 1}, {3, 27}};
  for (const SimtChoice& c : all)
    if (choice_valid(P, g, tk, sizeof(T), c)) cand.push_back(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(FMM_ERR_CUDA, "event creation failed");
  }
  fmm_status st = FMM_OK;
  float best = 1e30f;
  SimtChoice pick = *out;
  for (const SimtChoice& c : cand) {
    g.shape = c.shape;
    g.dsplit = c.dsplit;
    cudaError_t e = launch_nbr_gemm<T>(g, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_nbr_gemm<T>(g, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = fail(FMM_ERR_CUDA, "autotune launch failed: %s", cudaGetErrorString(e));
      break;
    }
    if (ms < best) best = ms, pick = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FMM_OK) return st;
  *out = pick;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = pick;
  return FMM_OK;
}

// Times the two tensor-core schedules of a contraction (3 launches after a
// warm-up each) and keeps the faster; cached per process like tune_one.
fmm_status tune_tc(fmm_plan_t P, int what, cudaStream_t s) {
  const bool tp = what == TS_M2L ? P->tp_m2l : what == TS_NEAR ? P->tp_near : P->tp_m2p;
  const bool span = what == TS_M2L ? P->span_m2l : what == TS_NEAR ? P->span_near : P->span_m2p;
  const bool ded = what == TS_NEAR && P->near4;  // the dedicated near-field kernel
  if ((int)tp + (int)span + (int)ded < 2) return FMM_OK;
  int level = P->L;  // M2L: the finest tensor-core level (the M2P's level excluded)
  if (what == TS_M2L) {
    level = -1;
    for (int l = 2; l <= P->L; ++l)
      if (P->lev[l].tc && !(l == P->L && P->m2p)) level = l;
    if (level < 0) return FMM_OK;
  }
  const int* g = what == TS_NEAR ? P->lev[P->L].n : P->lev[level].np;
  char key[160];
  std::snprintf(key, sizeof key, "tc%d/%d,%d,%d/%d/%d/%d/%d/%d", what, g[0], g[1], g[2], P->p, P->b, P->tc_kind,
                P->harm ? 1 : 0, P->near_comps);
  // candidate c: 0 span, 1 prefix, 2 the dedicated near-field kernel
  auto select = [&](int c) {
    P->use_tp[what] = c == 1;
    if (what == TS_NEAR) P->use_near4 = c == 2;
  };
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tc_tune_cache.find(key);
    if (it != g_tc_tune_cache.end()) {
      select(it->second);
      return FMM_OK;
    }
  }
  auto launch = [&]() -> fmm_status {
    if (what == TS_M2L) return do_m2l(P, level, s);
    if (what == TS_M2P) return do_m2p(P, s);
    return do_near_tc(P, s);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(FMM_ERR_CUDA, "event creation failed");
  }
  const bool have[3] = {span, tp, ded};
  float ms[3] = {0.f, 0.f, 0.f};
  int best = -1;
  fmm_status st = FMM_OK;
  for (int c = 0; c < 3 && st == FMM_OK; ++c) {
    if (!have[c]) continue;
    select(c);
    if ((st = launch())) break;  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(FMM_ERR_CUDA, "event record failed");
    for (int r = 0; r < 3 && st == FMM_OK; ++r) st = launch();
    if (st == FMM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms[c], e0, e1) != cudaSuccess))
      st = fail(FMM_ERR_CUDA, "tensor-core schedule timing failed");
    if (st == FMM_OK && (best < 0 || ms[c] < ms[best])) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FMM_OK) return st;
  select(best);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tc_tune_cache[key] = best;
  return FMM_OK;
}

}  // namespace

extern "C" fmm_status fmm_plan_autotune(fmm_plan_t P, void* stream) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // defined inputs for the timed launches; every solve rewrites the arena
  CUDA_TRY(cudaMemsetAsync(P->arena, 0, P->arena_bytes, s));
  fmm_status st;
  for (int l = 2; l <= P->L; ++l) {
    if (P->lev[l].tc) continue;
    const NbrGemm g = m2l_gemm(P, l);
    st = P->lev[l].f64 ? tune_one<double>(P, g, P->h_m2l_tile_k, "m2l", 3, s, &P->m2l_choice[l])
                       : tune_one<float>(P, g, P->h_m2l_tile_k, "m2l", 3, s, &P->m2l_choice[l]);
    if (st) return st;
  }
  if (!P->near_tc) {
    const NbrGemm g = near_gemm(P);
    st = P->f64_data() ? tune_one<double>(P, g, P->h_near_tile_k, "near", 3, s, &P->near_choice)
                       : tune_one<float>(P, g, P->h_near_tile_k, "near", 3, s, &P->near_choice);
    if (st) return st;
  }
  for (int what = 0; what < 3; ++what)
    if ((st = tune_tc(P, what, s))) return st;
  CUDA_TRY(cudaStreamSynchronize(s));
  return FMM_OK;
}

extern "C" fmm_status fmm_plan_tc_schedule(fmm_plan_t P, int what, int* prefix, int* available) {
  g_last_error.clear();
  if (!P || what < 0 || what > 2) return fail(FMM_ERR_ARG, "plan is NULL or `what` is not 0, 1 or 2");
  const bool tp = what == TS_M2L ? P->tp_m2l : what == TS_NEAR ? P->tp_near : P->tp_m2p;
  const bool span = what == TS_M2L ? P->span_m2l : what == TS_NEAR ? P->span_near : P->span_m2p;
  const bool ded = what == TS_NEAR && P->near4;
  if (available) *available = (span ? 1 : 0) | (tp ? 2 : 0) | (ded ? 4 : 0);
  if (prefix) *prefix = (ded && P->use_near4) ? 2 : (tp || span) ? (tc_prefix(P, what) ? 1 : 0) : -1;
  return FMM_OK;
}

extern "C" fmm_status fmm_plan_debug_timeout(fmm_plan_t P) {
  g_last_error.clear();
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  bool any = false;
  for (int l = 2; l <= P->L; ++l) any = any || (P->lev[l].tc && !(l == P->L && P->m2p));
  if (!any || !tc_prefix(P, TS_M2L)) return fail(FMM_ERR_ARG, "no M2L level of this plan runs the prefix schedule");
  P->inject_timeout = true;
  return FMM_OK;
}

extern "C" fmm_status fmm_plan_set_tc_schedule(fmm_plan_t P, int what, int prefix) {
  g_last_error.clear();
  if (!P || what < 0 || what > 2) return fail(FMM_ERR_ARG, "plan is NULL or `what` is not 0, 1 or 2");
  const bool tp = what == TS_M2L ? P->tp_m2l : what == TS_NEAR ? P->tp_near : P->tp_m2p;
  const bool span = what == TS_M2L ? P->span_m2l : what == TS_NEAR ? P->span_near : P->span_m2p;
  if (prefix == 2) {  // the dedicated near-field kernel
    if (what != TS_NEAR || !P->near4)
      return fail(FMM_ERR_ARG, "the dedicated kernel exists for the near field of leaf-4 potential plans only");
    P->use_near4 = true;
    return FMM_OK;
  }
  if (prefix < 0 || prefix > 2) return fail(FMM_ERR_ARG, "schedule must be 0 (span), 1 (prefix) or 2 (dedicated)");
  if (prefix ? !tp : !span) return fail(FMM_ERR_ARG, "the %s schedule of that contraction does not exist in this plan",
                                        prefix ? "prefix" : "span");
  if (what == TS_M2L && P->asym && !(prefix ? P->tp_m2l_t : P->span_m2l_t))
    return fail(FMM_ERR_ARG, "the transposed M2L has no %s schedule", prefix ? "prefix" : "span");
  P->use_tp[what] = prefix != 0;
  if (what == TS_NEAR) P->use_near4 = false;
  return FMM_OK;
}

namespace {
fmm_status tuning_slot(fmm_plan_t P, int level, SimtChoice** c, NbrGemm* g, const std::vector<int>** tk, size_t* es) {
  if (!P) return fail(FMM_ERR_ARG, "plan is NULL");
  if (level == -1) {
    if (P->near_tc) return fail(FMM_ERR_ARG, "the near field of this plan runs on the tensor cores");
    *c = &P->near_choice;
    *g = near_gemm(P);
    *tk = &P->h_near_tile_k;
    *es = P->esize();
    return FMM_OK;
  }
  if (level < 2 || level > P->L) return fail(FMM_ERR_ARG, "level %d outside 2..%d", level, P->L);
  if (P->lev[level].tc) return fail(FMM_ERR_ARG, "level %d runs on the tensor cores", level);
  *c = &P->m2l_choice[level];
  *g = m2l_gemm(P, level);
  *tk = &P->h_m2l_tile_k;
  *es = P->lev[level].f64 ? 8 : 4;
  return FMM_OK;
}
}  // namespace

extern "C" fmm_status fmm_plan_tuning(fmm_plan_t P, int level, int* shape, int* dsplit) {
  SimtChoice* c;
  NbrGemm g;
  const std::vector<int>* tk;
  size_t es;
  if (fmm_status st = tuning_slot(P, level, &c, &g, &tk, &es)) return st;
  if (shape) *shape = c->shape;
  if (dsplit) *dsplit = c->dsplit;
  return FMM_OK;
}

extern "C" fmm_status fmm_plan_set_tuning(fmm_plan_t P, int level, int shape, int dsplit) {
  SimtChoice* c;
  NbrGemm g;
  const std::vector<int>* tk;
  size_t es;
  if (fmm_status st = tuning_slot(P, level, &c, &g, &tk, &es)) return st;
  const SimtChoice want{shape, dsplit};
  if (!choice_valid(P, g, *tk, es, want))
    return fail(FMM_ERR_ARG, "variant shape %d / split %d does not apply to this contraction (or its split scratch "
                "does not fit the plan)", shape, dsplit);
  *c = want;
  return FMM_OK;
}
