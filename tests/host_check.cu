// Host-side checks of the plan's tables and tensor-core schedules (no GPU
// needed).  capi.cu, the library's host code, is compiled into this program.
//
//   host_check            the tensor-core schedules (below)
//   host_check plant      planted schedule corruptions, each must be caught
//   host_check tables DIR writes the plan's M2L, M2P and near-field weight
//                         tables and the kernels' M2M / L2L shifts of random
//                         expansions (FP64, raw) into DIR for comparison with
//                         the oracle's operators
//   host_check harmonic   harmonic compression against the Cartesian
//                         contraction, orders 2..8 (exact up to rounding)
//   host_check cuda-core  the CUDA-core M2L weight tiles (prefix-cut
//                         reductions) against the full contraction
//
// The library's plan packs every tensor-core contraction (M2L per level,
// final-stage M2P, the near field) into passes of MMA spans, per-issuer
// weight rings and pre-swizzled weight tiles.  This program builds those
// schedules with the library's own host code (capi.cu is compiled into it)
// and checks, for every order, precision and contraction kind:
//
//  * resources: a pass uses at most 512 TMEM columns, the weight rings are
//    1 KB multiples within the shared-memory budget;
//  * ownership: per chunk the issuers' span ranges are contiguous, every
//    accumulator column belongs to one issuer, an accumulator opens (its
//    first MMA overwrites) in one chunk only, by one span, and the epilogue
//    stores each output column from one group of one pass;
//  * the weight rings: replayed in the producer's order (tile, neighbour
//    column (dx, dz), chunk, dy, span) over two tiles, with the consumer
//    releasing spans only when the producer must wait, no span is larger than
//    its ring, every wait can be ended by a release, and live spans never
//    overlap in the ring;
//  * the arithmetic: the MMAs are emulated from the packed tiles (hi / lo
//    bf16 planes and swizzle, or TF32) over the 27 neighbour blocks of random
//    activations; the sum must cover every output column and equal the direct
//    contraction with the plan's weight function to the split precision's
//    rounding (bf16x3: 2e-5, TF32: 1e-3, of the sum of |terms|).
//
// Exit status 0 when every schedule passes; each case prints one line.
// With the argument "plant", it corrupts built schedules instead (a zeroed
// weight tile, a tile row read unswizzled, two issuers on one accumulator, an
// accumulator opened late, an accumulator opened by two spans, a ring smaller
// than a span) and exits 0 only if every corruption is caught.
#include "capi.cu"
#include "tree_common.cuh"

#include <cstdio>
#include <random>
#include <string>

namespace {

constexpr int kTiles = 2;  // the rings carry over from one tile to the next

uint32_t span_bytes(const TcSpan& S, int planes) { return (uint32_t)S.n * 128u * (S.prod ? 1u : (uint32_t)planes); }

// The byte ring of issuer q, as its producer fills it (virtual positions: v =
// start of the next span, last = end of the last span written, freed = end of
// the spans released).  Returns false on a span larger than the ring, a wait
// no release can end, or overlapping live spans.
bool ring_ok(const TcPass& P, int q, int planes) {
  const uint32_t RB = (uint32_t)P.ring_bytes[q];
  constexpr int E = 16;  // spans in flight per ring
  uint32_t beg_v[E], end_v[E], off_v[E];
  uint32_t e = 0, tail = 0, v = 0, off = 0, freed = 0, last = 0;
  for (int tile = 0; tile < kTiles; ++tile)
    for (int xz = 0; xz < 9; ++xz)
      for (int j = 0; j < P.nchunks; ++j)
        for (int dy = 0; dy < 3; ++dy)
          for (int si = P.span_idx[j][q]; si < P.span_idx[j][q + 1]; ++si) {
            const uint32_t bytes = span_bytes(P.span[si], planes);
            if (bytes > RB) return false;
            if (off + bytes > RB) v += RB - off, off = 0;  // a span never wraps
            const uint32_t need = v + bytes > RB ? std::min(last, v + bytes - RB) : 0u;
            while (freed < need || e - tail >= (uint32_t)E) {
              if (tail == e) return false;  // nothing left to release
              freed = end_v[tail % E];
              ++tail;
            }
            for (uint32_t t = tail; t < e; ++t) {  // live spans must not overlap the new one
              const uint32_t o = off_v[t % E], b = end_v[t % E] - beg_v[t % E];
              if (o < off + bytes && off < o + b) return false;
            }
            beg_v[e % E] = v;
            off_v[e % E] = off;
            end_v[e % E] = v + bytes;
            v += bytes;
            last = v;
            off += bytes;
            ++e;
          }
  return true;
}

// Output group and column of TMEM column tcol in pass P, or g = -1.
void tmem_owner(const TcPass& P, int tcol, int& g, int& c) {
  g = c = -1;
  for (int q = 0; q < P.ng; ++q) {
    const int acc[4] = {P.out_tmem[q], P.out_tmem2[q], P.out_tmem3[q], P.out_tmem4[q]};
    for (int a : acc)
      if (a >= 0 && tcol >= a && tcol < a + P.out_nmma[q]) g = q, c = tcol - a;
  }
}

float tf32_trunc(float a) {  // the tensor cores read FP32 operands as TF32
  uint32_t u;
  std::memcpy(&u, &a, 4);
  u &= ~0x1FFFu;
  std::memcpy(&a, &u, 4);
  return a;
}

bool fail(const char* name, const char* what, int pass) {
  std::printf("%s: FAILED (%s, pass %d)\n", name, what, pass);
  return false;
}

// ncol output columns, klen reduction values per neighbour block;
// entry(d, k, n) is the weight the schedule must reproduce.
template <typename Entry>
bool check(const char* name, int kind, const TcHost& H, int ncol, int klen, const Entry& entry) {
  const int chunk = kind == TC_BF16X3 ? 64 : 32, kstep = chunk / 4, esz = kind == TC_BF16X3 ? 2 : 4;
  const int planes = kind == TC_BF16X3 ? 2 : 1;
  std::mt19937 rng(ncol * 3 + kind);
  std::uniform_real_distribution<double> U(-1, 1);
  std::vector<std::vector<float>> A(27, std::vector<float>(klen, 0.f));
  for (auto& r : A)
    for (float& a : r) a = (float)U(rng);
  std::vector<double> ref(ncol, 0), got(ncol, 0), sabs(ncol, 0);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < klen; ++k)
      for (int n = 0; n < ncol; ++n) {
        const double t = A[d][k] * entry(d, k, n);
        ref[n] += t;
        sabs[n] += std::fabs(t);
      }
  std::vector<int> covered(ncol, 0), writer(ncol, -1);
  int spans = 0;
  for (int ps = 0; ps < H.npass; ++ps) {
    const TcPass& P = H.pass[ps];
    spans += P.span_idx[P.nchunks][0];
    // the epilogue stores each output column once: one group of one pass
    for (int g = 0; g < P.ng; ++g)
      for (int c = 0; c < P.out_ncols[g]; ++c) {
        const int n = P.out_col0[g] + c;
        if (n < 0 || n >= ncol) return fail(name, "output column out of range", ps);
        if (writer[n] >= 0) return fail(name, "output column stored by two groups", ps);
        writer[n] = ps * 64 + g;
      }
    if (P.tmem_cols > 512) return fail(name, "more than 512 TMEM columns", ps);
    long ring_sum = 0;
    for (int q = 0; q < kTcIssuers; ++q) {
      if (P.ring_bytes[q] % 1024) return fail(name, "ring not a 1 KB multiple", ps);
      ring_sum += P.ring_bytes[q];
    }
    if (ring_sum > tc_ring_budget(kind, H.a_stages)) return fail(name, "rings over the budget", ps);
    std::vector<int> owner(512, -1), opened(512, -1);
    for (int j = 0; j < P.nchunks; ++j) {
      if (P.span_idx[j][kTcIssuers] != P.span_idx[j + 1][0]) return fail(name, "span ranges not contiguous", ps);
      // in the chunk where an accumulator opens, one span only may write it
      // (every span of that chunk's first step overwrites)
      std::vector<int> openers(512, 0);
      for (int si = P.span_idx[j][0]; si < P.span_idx[j][kTcIssuers]; ++si)
        if (P.span[si].first == j)
          for (int r = 0; r < P.span[si].n; ++r)
            if (++openers[P.span[si].tmem_col + r] > 1) return fail(name, "accumulator opened by two spans", ps);
      for (int q = 0; q < kTcIssuers; ++q) {
        if (P.span_idx[j][q] > P.span_idx[j][q + 1]) return fail(name, "span range reversed", ps);
        for (int si = P.span_idx[j][q]; si < P.span_idx[j][q + 1]; ++si) {
          const TcSpan& S = P.span[si];
          if (S.n % 16 || S.n > 192 || S.ksteps < 1 || S.ksteps > 4) return fail(name, "bad MMA shape", ps);
          for (int r = 0; r < S.n; ++r) {
            int& o = owner[S.tmem_col + r];
            if (o >= 0 && o != q) return fail(name, "TMEM column shared by two issuers", ps);
            o = q;
            int& op = opened[S.tmem_col + r];
            if (op < 0) {
              if (S.first != j) return fail(name, "accumulator opened after its first MMA", ps);
              op = j;
            } else if (S.first != op) {
              return fail(name, "accumulator opened twice", ps);
            }
          }
        }
      }
    }
    for (int q = 0; q < kTcIssuers; ++q)
      if (!ring_ok(P, q, planes)) return fail(name, "weight ring stalls or overlaps", ps);
    for (int g = 0; g < P.ng; ++g)
      for (int c = 0; c < P.out_nmma[g]; ++c) {
        const int acc[4] = {P.out_tmem[g], P.out_tmem2[g], P.out_tmem3[g], P.out_tmem4[g]};
        for (int a : acc)
          if (a >= 0 && owner[a + c] < 0) return fail(name, "epilogue reads an unwritten accumulator", ps);
      }
    // emulate every MMA of the pass on one row (a parent, or a leaf box)
    for (int d = 0; d < 27; ++d)
      for (int j = 0; j < P.nchunks; ++j)
        for (int si = P.span_idx[j][0]; si < P.span_idx[j][kTcIssuers]; ++si) {
          const TcSpan& S = P.span[si];
          const unsigned char* tile = H.W.data() + P.w_base + (size_t)d * P.bytes_per_d + S.w_off;
          for (int r = 0; r < S.n; ++r) {
            int g, c;
            tmem_owner(P, S.tmem_col + r, g, c);
            if (g < 0) return fail(name, "span writes outside every accumulator", ps);
            if (c >= P.out_ncols[g]) continue;  // padding column
            const int n = P.out_col0[g] + c;
            covered[n] = 1;
            for (int e = 0; e < S.ksteps * kstep; ++e) {
              const int k = j * chunk + e;
              const float a = k < klen ? A[d][k] : 0.f;
              const int byte = e * esz;  // 128-byte rows, 16-byte chunks swizzled by (row mod 8)
              const size_t off = (size_t)r * 128 + (size_t)((((byte >> 4) ^ (r & 7)) << 4) | (byte & 15));
              if (kind == TC_BF16X3) {
                const float ah = bf16_to_f(bf16_rn(a)), al = bf16_to_f(bf16_rn(a - ah));
                uint16_t w1;
                std::memcpy(&w1, tile + off, 2);
                if (S.prod == 0) {  // hi and lo planes, three products
                  uint16_t wl;
                  std::memcpy(&wl, tile + (size_t)S.n * 128 + off, 2);
                  got[n] += (double)ah * bf16_to_f(w1) + (double)ah * bf16_to_f(wl) + (double)al * bf16_to_f(w1);
                } else {
                  got[n] += (double)(S.prod == 3 ? al : ah) * bf16_to_f(w1);
                }
              } else {
                float w;
                std::memcpy(&w, tile + off, 4);
                got[n] += (double)tf32_trunc(a) * w;
              }
            }
          }
        }
  }
  double err = 0;
  int missing = 0;
  for (int n = 0; n < ncol; ++n) {
    missing += !covered[n];
    if (sabs[n] > 0) err = std::max(err, std::fabs(got[n] - ref[n]) / sabs[n]);
  }
  const double tol = kind == TC_BF16X3 ? 2e-5 : 1e-3;
  std::printf("%-28s %-6s passes %d spans %3d weights %6.2f MB uncovered %d err/sum|terms| %.2e\n", name,
              kind == TC_BF16X3 ? "bf16x3" : "tf32", H.npass, spans, H.W.size() / 1e6, missing, err);
  if (missing) return fail(name, "output columns never written", -1);
  if (!(err <= tol)) return fail(name, "result differs from the direct contraction", -1);
  return true;
}

// mult_order / local_order: -1 for the order itself
bool m2l_case(int kind, int p, int mult_order, int local_order, bool harm) {
  MultiIndex mi;
  mi.init(p);
  if (mult_order >= 0) mi.mo = mult_order;
  if (local_order >= 0) mi.lo = local_order;
  TaylorTable tt;
  tt.build(mi);
  TcHost H;
  char name[64];
  std::snprintf(name, sizeof name, "m2l p=%d mo=%d lo=%d%s", p, mi.mo, mi.lo, harm ? " harmonic" : "");
  if (!build_tc(mi, tt, kind, H, harm)) return fail(name, "schedule not built", -1);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  return check(name, kind, H, 8 * nk, 8 * nk, [&](int d, int k, int n) {
    return harm ? m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8) : m2l_entry(mi, tt, d, k, n);
  });
}

bool m2p_case(int kind, int p, int b, int mult_order, bool harm) {
  MultiIndex mi;
  mi.init(p);
  if (mult_order >= 0) mi.mo = mult_order;
  M2pTable tab;
  tab.build(mi, b);
  TcHost H;
  char name[64];
  std::snprintf(name, sizeof name, "m2p p=%d mo=%d b=%d%s", p, mi.mo, b, harm ? " harmonic" : "");
  if (!build_tc_m2p(mi, tab, kind, H, harm)) return fail(name, "schedule not built", -1);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  return check(name, kind, H, 8 * b * b * b, 8 * nk, [&](int d, int k, int n) {
    return harm ? m2p_entry(mi, tab, d, red[k / 8] * 8 + k % 8, n) : m2p_entry(mi, tab, d, k, n);
  });
}

bool near_case(int b, int comps) {
  TcHost H;
  char name[64];
  std::snprintf(name, sizeof name, "near b=%d columns=%d", b, comps);
  if (!build_tc_near(b, comps, TC_BF16X3, H)) return fail(name, "schedule not built", -1);
  return check(name, TC_BF16X3, H, comps * b * b * b, b * b * b, [b](int d, int k, int n) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    return near_entry(b, D, k, n);
  });
}

// Planted mistakes: each corrupts one built schedule (order 6, harmonic,
// bf16x3) and must be caught.  Returns the number that were not.
int planted_mistakes() {
  MultiIndex mi;
  mi.init(6);
  TaylorTable tt;
  tt.build(mi);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = (int)red.size();
  auto entry = [&](int d, int k, int n) { return m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8); };
  int missed = 0;
  auto plant = [&](const char* what, auto corrupt) {
    TcHost H;
    if (!build_tc(mi, tt, TC_BF16X3, H, true) || !corrupt(H)) {
      std::printf("planted mistake could not be placed: %s\n", what);
      ++missed;
      return;
    }
    if (check(what, TC_BF16X3, H, 8 * nk, 8 * nk, entry)) {
      std::printf("planted mistake NOT caught: %s\n", what);
      ++missed;
    }
  };
  // first span of issuer q in pass 0, or -1
  auto first_span = [](const TcPass& P, int q) {
    for (int j = 0; j < P.nchunks; ++j)
      if (P.span_idx[j][q] < P.span_idx[j][q + 1]) return P.span_idx[j][q];
    return -1;
  };
  plant("zeroed weight tile", [](TcHost& H) {  // neighbour 0 (a corner parent): non-zero weights
    const TcPass& P = H.pass[0];
    std::fill_n(H.W.begin() + P.w_base + P.span[0].w_off, (size_t)P.span[0].n * 128 * 2, (unsigned char)0);
    return true;
  });
  plant("tile row read unswizzled", [](TcHost& H) {  // row 1: its 16-byte chunks 0 and 1 trade places
    const TcPass& P = H.pass[0];
    unsigned char* row = H.W.data() + P.w_base + P.span[0].w_off + 128;
    std::swap_ranges(row, row + 16, row + 16);
    return true;
  });
  plant("two issuers on one accumulator", [&](TcHost& H) {
    TcPass& P = H.pass[0];
    const int a = first_span(P, 0), b = first_span(P, 1);
    if (a < 0 || b < 0) return false;
    P.span[b].tmem_col = P.span[a].tmem_col;
    return true;
  });
  plant("accumulator opened one chunk late", [](TcHost& H) {
    TcPass& P = H.pass[0];
    if (P.nchunks < 2) return false;
    P.span[P.span_idx[0][0]].first = 1;
    return true;
  });
  plant("accumulator opened by two spans", [](TcHost& H) {  // two openers of one issuer in one chunk
    TcPass& P = H.pass[0];
    for (int j = 0; j < P.nchunks; ++j)
      for (int q = 0; q < kTcIssuers; ++q) {
        int a = -1;
        for (int si = P.span_idx[j][q]; si < P.span_idx[j][q + 1]; ++si) {
          if (P.span[si].first != j) continue;
          if (a < 0) {
            a = si;
          } else {
            P.span[si].tmem_col = P.span[a].tmem_col;
            return true;
          }
        }
      }
    return false;
  });
  plant("weight ring smaller than a span", [](TcHost& H) {
    H.pass[0].ring_bytes[0] = 1024;
    return true;
  });
  return missed;
}

// ---------------------------------------------------------------- tables --

bool write_table(const std::string& path, const std::vector<double>& v) {
  FILE* f = std::fopen(path.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(v.data(), sizeof(double), v.size(), f) == v.size();
  return std::fclose(f) == 0 && ok;
}

// M2L weights [27][8 nc][8 nc] (neighbour parent, alpha*8 + source child,
// beta*8 + target child) with multipole / local limits mo, lo.
bool dump_m2l(const std::string& dir, int p, int mo, int lo) {
  MultiIndex mi;
  mi.init(p);
  mi.mo = mo, mi.lo = lo;
  TaylorTable tt;
  tt.build(mi);
  const int K = 8 * mi.nc;
  std::vector<double> W((size_t)27 * K * K);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < K; ++k)
      for (int n = 0; n < K; ++n) W[((size_t)d * K + k) * K + n] = m2l_entry(mi, tt, d, k, n);
  char name[64];
  std::snprintf(name, sizeof name, "/m2l_p%d_mo%d_lo%d.bin", p, mo, lo);
  return write_table(dir + name, W);
}

// Final-stage M2P weights [27][8 nc][8 b^3] (neighbour parent, alpha*8 +
// source child, target child * b^3 + cell).
bool dump_m2p(const std::string& dir, int p, int b) {
  MultiIndex mi;
  mi.init(p);
  M2pTable tab;
  tab.build(mi, b);
  const int K = 8 * mi.nc, N = 8 * b * b * b;
  std::vector<double> W((size_t)27 * K * N);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < K; ++k)
      for (int n = 0; n < N; ++n) W[((size_t)d * K + k) * N + n] = m2p_entry(mi, tab, d, k, n);
  char name[64];
  std::snprintf(name, sizeof name, "/m2p_p%d_b%d.bin", p, b);
  return write_table(dir + name, W);
}

// Near-field weights [27][b^3][4 b^3] (neighbour box, source cell,
// component * b^3 + target cell; components: g, then the three force columns).
bool dump_near(const std::string& dir, int b) {
  const int b3 = b * b * b;
  std::vector<double> W((size_t)27 * b3 * 4 * b3);
  for (int d = 0; d < 27; ++d) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    for (int k = 0; k < b3; ++k)
      for (int n = 0; n < 4 * b3; ++n) W[((size_t)d * b3 + k) * 4 * b3 + n] = near_entry(b, D, k, n);
  }
  char name[64];
  std::snprintf(name, sizeof name, "/near_b%d.bin", b);
  return write_table(dir + name, W);
}

// ---------------------------------------------------------------- shifts --

// The kernels' separable shifts (M2M: shift_up, L2L: shift_down along x, y,
// z in turn) for random expansions and displacements; each case is written as
// [input (nc), d (3), output (nc)] for comparison with the oracle's M2M / L2L.
template <int P>
bool dump_shifts(const std::string& dir) {
  constexpr int NC = fmmgb::tree::ncoef_c(P);
  std::mt19937 rng(300 + P);
  std::uniform_real_distribution<double> U(-1, 1);
  std::vector<double> up, down;
  for (int rep = 0; rep < 6; ++rep) {
    double M[NC], L[NC], d[3], dp[P + 1];
    for (int k = 0; k < NC; ++k) M[k] = U(rng), L[k] = U(rng);
    for (double& x : d) x = U(rng);
    if (rep == 0) d[0] = fmmgb::tree::half_offset<double>(5, 0), d[1] = fmmgb::tree::half_offset<double>(5, 1),
                  d[2] = fmmgb::tree::half_offset<double>(5, 2);  // a child offset, as the kernels use
    up.insert(up.end(), M, M + NC);
    up.insert(up.end(), d, d + 3);
    down.insert(down.end(), L, L + NC);
    down.insert(down.end(), d, d + 3);
    fmmgb::tree::powers<P, double>(d[0], dp);
    fmmgb::tree::shift_up<P, 0, double>(M, dp);
    fmmgb::tree::shift_down<P, 0, double>(L, dp);
    fmmgb::tree::powers<P, double>(d[1], dp);
    fmmgb::tree::shift_up<P, 1, double>(M, dp);
    fmmgb::tree::shift_down<P, 1, double>(L, dp);
    fmmgb::tree::powers<P, double>(d[2], dp);
    fmmgb::tree::shift_up<P, 2, double>(M, dp);
    fmmgb::tree::shift_down<P, 2, double>(L, dp);
    up.insert(up.end(), M, M + NC);
    down.insert(down.end(), L, L + NC);
  }
  char a[64], b[64];
  std::snprintf(a, sizeof a, "/shift_up_p%d.bin", P);
  std::snprintf(b, sizeof b, "/shift_down_p%d.bin", P);
  return write_table(dir + a, up) && write_table(dir + b, down);
}

// ------------------------------------------------------ CUDA-core tiles --

// The CUDA-core M2L weight tiles (32 output columns each, reduction cut to
// the prefix the tile's lowest order needs): the contraction read from the
// tiles as the kernels read it must equal the full contraction with the
// weight function, i.e. no non-zero weight lies past a tile's prefix.
bool cc_tiles_case(int p, int mo, int lo, bool harm) {
  MultiIndex mi;
  mi.init(p);
  if (mo >= 0) mi.mo = mo;
  if (lo >= 0) mi.lo = lo;
  TaylorTable tt;
  tt.build(mi);
  std::vector<double> W;
  std::vector<int> tk;
  std::vector<long long> tw;
  m2l_weights<double>(mi, tt, W, tk, tw, true, harm);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc, K = 8 * nk, ncol = 8 * nk;
  std::mt19937 rng(500 + p);
  std::uniform_real_distribution<double> U(-1, 1);
  std::vector<std::vector<double>> A(27, std::vector<double>(K));
  for (auto& r : A)
    for (double& a : r) a = U(rng);
  double err = 0;
  long long kept = 0, full = 0;
  for (int n = 0; n < ncol; ++n) {
    const int t = n / kNTile, j = n % kNTile;
    double got = 0, ref = 0, sabs = 0;
    for (int d = 0; d < 27; ++d) {
      const double* blk = W.data() + tw[t] + (long long)d * tk[t] * kNTile;
      for (int k = 0; k < tk[t]; ++k) got += A[d][k] * blk[(long long)k * kNTile + j];
      for (int k = 0; k < K; ++k) {
        const double w = harm ? m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8)
                              : m2l_entry(mi, tt, d, k, n);
        ref += A[d][k] * w;
        sabs += std::fabs(A[d][k] * w);
      }
      kept += tk[t];
      full += K;
    }
    if (sabs > 0) err = std::max(err, std::fabs(got - ref) / sabs);
  }
  std::printf("cuda-core tiles p=%d mo=%d lo=%d%s: reduction kept %.0f%%, err/sum|terms| %.1e\n", p, mi.mo, mi.lo,
              harm ? " harmonic" : "", 100.0 * kept / full, err);
  return err <= 1e-13;
}

int cc_tiles_check() {
  int bad = 0;
  for (int p = 2; p <= 8; ++p)
    for (bool harm : {false, true}) bad += !cc_tiles_case(p, -1, -1, harm);
  for (bool harm : {false, true}) {
    bad += !cc_tiles_case(3, 2, -1, harm);  // the paper's orders
    bad += !cc_tiles_case(3, -1, 2, harm);  // and their transpose
    bad += !cc_tiles_case(6, 4, -1, harm);
  }
  return bad;
}

// ------------------------------------------------------------- harmonic --

// For random multipoles of one source child, the compressed contraction
// (fold the multipoles, contract the (p+1)^2 components with the reduced
// weights, rebuild the locals with c >= 2) must equal the Cartesian one, for
// every neighbour parent and child pair.  The same for M2P (fold only).
template <int P>
double harmonic_error() {
  constexpr int NC = fmmgb::tree::ncoef_c(P);
  MultiIndex mi;
  mi.init(P);
  TaylorTable tt;
  tt.build(mi);
  M2pTable tab;
  tab.build(mi, 2);
  const std::vector<int> red = harmonic_components(mi);
  std::mt19937 rng(100 + P);
  std::uniform_real_distribution<double> U(-1, 1);
  double err = 0;
  for (int d = 0; d < 27; ++d)
    for (int cs = 0; cs < 8; ++cs) {
      double M[NC], Mf[NC];
      for (int k = 0; k < NC; ++k) Mf[k] = M[k] = U(rng);
      fmmgb::tree::harmonic_fold<P, double>(Mf);
      for (int ct = 0; ct < 8; ++ct) {
        double Lc[NC] = {}, Lh[NC] = {}, scale = 0;
        for (int n = 0; n < NC; ++n)
          for (int k = 0; k < NC; ++k) {
            const double w = m2l_entry(mi, tt, d, k * 8 + cs, n * 8 + ct);
            Lc[n] += w * M[k];
            scale += std::fabs(w * M[k]);
          }
        for (int rn : red)
          for (int rk : red) Lh[rn] += m2l_entry(mi, tt, d, rk * 8 + cs, rn * 8 + ct) * Mf[rk];
        fmmgb::tree::harmonic_expand<P, double>(Lh);
        for (int n = 0; n < NC; ++n) err = std::max(err, std::fabs(Lh[n] - Lc[n]) / std::max(scale, 1e-300));
        for (int cell = 0; cell < 8; ++cell) {
          const int col = ct * 8 + cell;
          double pc = 0, ph = 0, s2 = 0;
          for (int k = 0; k < NC; ++k) {
            const double w = m2p_entry(mi, tab, d, k * 8 + cs, col);
            pc += w * M[k];
            s2 += std::fabs(w * M[k]);
          }
          for (int rk : red) ph += m2p_entry(mi, tab, d, rk * 8 + cs, col) * Mf[rk];
          err = std::max(err, std::fabs(ph - pc) / std::max(s2, 1e-300));
        }
      }
    }
  return err;
}

// The L2L kernel adds the M2L's c <= 1 locals to the parent's shifted
// locals and rebuilds the c >= 2 components of the sum in place.  That needs
// the shifted parent locals to be harmonic themselves: a harmonic local
// expansion (c >= 2 rebuilt from c <= 1) shifted by shift_down along x, y, z
// must equal the rebuild of its own c <= 1 part.
template <int P>
double harmonic_shift_error() {
  constexpr int NC = fmmgb::tree::ncoef_c(P);
  MultiIndex mi;
  mi.init(P);
  const std::vector<int> red = harmonic_components(mi);
  std::mt19937 rng(700 + P);
  std::uniform_real_distribution<double> U(-1, 1);
  double err = 0;
  for (int rep = 0; rep < 16; ++rep) {
    double L[NC] = {}, R[NC], dp[P + 1];
    for (int k : red) L[k] = U(rng);
    fmmgb::tree::harmonic_expand<P, double>(L);
    for (int q = 0; q < 3; ++q) {
      fmmgb::tree::powers<P, double>(fmmgb::tree::half_offset<double>(rep & 7, q), dp);
      if (q == 0) fmmgb::tree::shift_down<P, 0, double>(L, dp);
      if (q == 1) fmmgb::tree::shift_down<P, 1, double>(L, dp);
      if (q == 2) fmmgb::tree::shift_down<P, 2, double>(L, dp);
    }
    for (int k = 0; k < NC; ++k) R[k] = 0;
    for (int k : red) R[k] = L[k];
    fmmgb::tree::harmonic_expand<P, double>(R);
    double scale = 0;
    for (int k = 0; k < NC; ++k) scale = std::max(scale, std::fabs(L[k]));
    for (int k = 0; k < NC; ++k) err = std::max(err, std::fabs(R[k] - L[k]) / scale);
  }
  return err;
}

int harmonic_check() {
  const double shift_errs[7] = {harmonic_shift_error<2>(), harmonic_shift_error<3>(), harmonic_shift_error<4>(),
                                harmonic_shift_error<5>(), harmonic_shift_error<6>(), harmonic_shift_error<7>(),
                                harmonic_shift_error<8>()};
  int bad_shift = 0;
  for (int p = 2; p <= 8; ++p) {
    std::printf("harmonic locals stay harmonic under L2L, p=%d: %.2e\n", p, shift_errs[p - 2]);
    bad_shift += !(shift_errs[p - 2] <= 1e-13);
  }
  if (bad_shift) return bad_shift;
  const double errs[7] = {harmonic_error<2>(), harmonic_error<3>(), harmonic_error<4>(), harmonic_error<5>(),
                          harmonic_error<6>(), harmonic_error<7>(), harmonic_error<8>()};
  int bad = 0;
  for (int p = 2; p <= 8; ++p) {
    std::printf("harmonic p=%d: max |compressed - Cartesian| / sum|terms| = %.2e\n", p, errs[p - 2]);
    bad += !(errs[p - 2] <= 1e-12);
  }
  return bad;
}

}  // namespace

int main(int argc, char** argv) {
  const std::string mode = argc > 1 ? argv[1] : "";
  if (mode == "plant") return planted_mistakes() ? 1 : 0;
  if (mode == "harmonic") return harmonic_check() ? 1 : 0;
  if (mode == "cuda-core") return cc_tiles_check() ? 1 : 0;
  if (mode == "tables") {
    if (argc < 3) return 2;
    const std::string dir = argv[2];
    const bool ok = dump_m2l(dir, 3, 3, 3) && dump_m2l(dir, 4, 4, 4) && dump_m2l(dir, 4, 3, 4) &&
                    dump_m2l(dir, 4, 4, 3) && dump_m2p(dir, 3, 2) && dump_m2p(dir, 4, 4) && dump_near(dir, 2) &&
                    dump_near(dir, 4) && dump_shifts<3>(dir) && dump_shifts<6>(dir) && dump_shifts<8>(dir);
    return ok ? 0 : 1;
  }
  bool ok = true;
  for (int kind : {TC_BF16X3, TC_TF32})
    for (int p : {2, 4, 6, 8})
      for (bool harm : {false, true}) ok &= m2l_case(kind, p, -1, -1, harm);
  for (int p : {3, 4, 6})  // multipoles below the order; the transpose: locals below it
    for (bool harm : {false, true}) {
      ok &= m2l_case(TC_BF16X3, p, p - 1, -1, harm);
      ok &= m2l_case(TC_BF16X3, p, -1, p - 1, harm);
      ok &= m2p_case(TC_BF16X3, p, 2, p - 1, harm);
    }
  for (int kind : {TC_BF16X3, TC_TF32})
    for (int p : {4, 6})
      for (int b : {2, 4})
        for (bool harm : {false, true}) ok &= m2p_case(kind, p, b, -1, harm);
  for (int b : {4, 8})
    for (int comps : {1, 4}) ok &= near_case(b, comps);
  return ok ? 0 : 1;
}
