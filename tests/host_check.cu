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
//   host_check prefix     the prefix-schedule contractions (k_nbr_tc.cu):
//                         resources, owner rings, one writer per TMEM
//                         column, emulated MMAs, randomised protocol replays
//   host_check prefix-plant  planted prefix-schedule mistakes, each caught
//   host_check rounding   the FP32 accumulation-chain bound of each schedule
//   host_check batch fp32|fp64 ORDER LEAF NX NY NZ [NX NY NZ ...]
//                         the fused batch's launch and item tables for fields
//                         of those grids (layout-only plans, no GPU)
//   host_check batch-plant ...  planted table corruptions, each caught
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
#include "multi.cuh"
#include "tree_common.cuh"

#include <array>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cmath>
#include <functional>
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

// ------------------------------------------------------- prefix schedule --
//
// The prefix schedules (k_nbr_tc.cu, build_tp_*): resources (TMEM columns of
// the accumulator sets, ring slots against the producer lanes, piece sizes),
// the program's fields (every MMA inside its piece and inside its accumulator
// set, N a multiple of 16 up to 256, pieces never crossing a chunk), the
// epilogue's groups (D, reversed E and L2 regions inside the set), and the
// arithmetic: every MMA emulated from the packed, swizzled 32-byte rows
// (bf16 hi / lo planes or TF32) over the 27 neighbour rows of random
// activations, accumulated per TMEM column and read back the epilogue's way,
// against the direct contraction.  `rz` also accumulates every MMA's sum into
// FP32 with truncation (the tensor cores' adder) on same-signed activations,
// to compare accumulator chains between schedules.

// The kernel's barrier protocol replayed on the CPU (the same slot, stage and
// parity arithmetic as k_nbr_tc.cu): activation producer groups, one weight
// producer per owner ring, the issuers (every stage, their own pieces), the
// epilogue's accumulator hand-off.  A barrier is a count of completed phases
// plus the arrivals of the current one; a wait is modelled as the hardware
// does it (satisfied when the current phase's parity differs from the one
// waited for) and must agree with the phase the protocol means; each run
// picks the next actor at random, and every actor must finish.
struct SimBar {
  int expected = 1, arrived = 0, done = 0;  // done: completed phases
  void arrive(int n = 1) {
    arrived += n;
    while (arrived >= expected) arrived -= expected, ++done;
  }
  bool hw(uint32_t parity) const { return (uint32_t)(done & 1) != parity; }
};

std::string simulate_protocol(const TpHost& H, int kind, int nitems, unsigned seed) {
  const int planes = kind == TC_BF16X3 ? 2 : 1, G = kTpALanes / planes, nA = H.a_stages, Q = kTpIssuers;
  std::vector<SimBar> a_full(nA), a_empty(nA), w_full(H.w_slots), w_empty(H.w_slots), acc_full(2), acc_empty(2);
  for (auto& b : a_full) b.expected = planes;
  for (auto& b : a_empty) b.expected = Q;
  for (auto& b : acc_full) b.expected = Q;
  for (auto& b : acc_empty) b.expected = 4;
  // the work each CTA does: items of passes (item i -> pass i % npass), as a flat list of stages
  struct Stage { int pass, xz, j; };
  std::vector<std::vector<Stage>> item_stages(nitems);
  std::vector<int> item_pass(nitems);
  for (int it = 0; it < nitems; ++it) {
    item_pass[it] = it * (int)H.pass.size() / nitems;
    for (int xz = 0; xz < 9; ++xz)
      for (int j = 0; j < H.pass[item_pass[it]].nchunks; ++j) item_stages[it].push_back({item_pass[it], xz, j});
  }
  std::vector<Stage> stages;
  for (auto& v : item_stages) stages.insert(stages.end(), v.begin(), v.end());
  const int T = (int)stages.size();
  // owner piece sequences (owner-local index l -> (stage, piece))
  std::vector<std::vector<std::pair<int, int>>> own(Q);
  for (int t = 0; t < T; ++t) {
    const TpPass& P = H.pass[stages[t].pass];
    for (int k = P.chunk_piece[stages[t].j]; k < P.chunk_piece[stages[t].j + 1]; ++k) own[P.piece_owner[k]].push_back({t, k});
  }
  auto acc_buf = [&](int it, std::vector<int>& uses, int& flip, int& phase) {
    const int nbuf = H.pass[item_pass[it]].nbuf;
    const int buf = nbuf == 2 ? (flip++ & 1) : 0;
    phase = uses[buf]++;
    return buf;
  };
  std::mt19937 rng(seed);
  std::string err;
  auto wait_ok = [&](const SimBar& b, int phase_index, uint32_t parity, const char* who) {
    const bool intended = b.done > phase_index, hardware = b.hw(parity);
    if (intended != hardware && err.empty())
      err = std::string(who) + ": a parity wait that does not match its phase (" +
            (hardware ? "passes early" : "would hang") + ")";
    return intended && hardware;
  };
  // actors
  std::vector<int> a_next(G, 0);               // next stage of A group g
  std::vector<size_t> w_next(Q, 0);            // next owner-local piece of producer q
  struct Iss { int item = 0, t = 0, stage_in_item = 0, piece = -1, phase = 0, buf = 0, state = 0; size_t l = 0;
               std::vector<int> uses{0, 0}; int flip = 0; };
  std::vector<Iss> iss(Q);
  struct Epi { int item = 0, state = 0, buf = 0, phase = 0; std::vector<int> uses{0, 0}; int flip = 0; } epi;
  // each actor's speed for this run: skewed interleavings (an idle issuer far
  // ahead of a busy one) are the ones that expose a mis-sequenced wait
  std::vector<double> speed(G + 2 * Q + 1);
  for (double& v : speed) v = std::pow(10.0, (double)(rng() % 3));
  auto pick = [&](const std::vector<int>& c) {
    double tot = 0;
    for (int a : c) tot += speed[a];
    double r = tot * (rng() / (double)rng.max());
    for (int a : c)
      if ((r -= speed[a]) <= 0) return a;
    return c.back();
  };
  for (auto& g : a_next) g = 0;
  for (int g = 0; g < G; ++g) while (a_next[g] < T && (a_next[g] % nA) % G != g) ++a_next[g];
  acc_empty[0].arrive(4);
  acc_empty[1].arrive(4);
  for (int step = 0; step < 50000000 && err.empty(); ++step) {
    std::vector<int> can;  // actors that can move: 0..G-1 A groups, G..G+Q-1 producers, G+Q.. issuers, last epilogue
    auto try_actor = [&](int a, bool act) -> bool {
      if (a < G) {
        const int t = a_next[a];
        if (t >= T) return false;
        const int slot = t % nA, use = t / nA;
        if (use > 0 && !wait_ok(a_empty[slot], use - 1, ((use & 1) ^ 1), "activation producer")) return false;
        if (act) {
          a_full[slot].arrive(planes);
          int nt = t + 1;
          while (nt < T && (nt % nA) % G != a) ++nt;
          a_next[a] = nt;
        }
        return true;
      }
      if (a < G + Q) {
        const int q = a - G;
        const size_t l = w_next[q];
        if (l >= own[q].size()) return false;
        const int ns = H.owner_nslots[q], slot = H.owner_slot0[q] + (int)(l % ns), use = (int)(l / ns);
        if (use > 0 && !wait_ok(w_empty[slot], use - 1, ((use & 1) ^ 1), "weight producer")) return false;
        if (act) w_full[slot].arrive(), ++w_next[q];
        return true;
      }
      if (a < G + 2 * Q) {
        const int q = a - G - Q;
        Iss& I = iss[q];
        if (I.item >= nitems) return false;
        const TpPass& P = H.pass[item_pass[I.item]];
        if (I.state == 0) {  // accumulator set
          int flip = I.flip, ph = 0;
          std::vector<int> uses = I.uses;
          const int buf = acc_buf(I.item, uses, flip, ph);
          if (!wait_ok(acc_empty[buf], ph, ph & 1, "issuer (accumulators)")) return false;
          if (act) I.flip = flip, I.uses = uses, I.buf = buf, I.state = 1;
          return true;
        }
        if (I.state == 1) {  // stage t
          const int slot = I.t % nA, use = I.t / nA;
          if (!wait_ok(a_full[slot], use, use & 1, "issuer (activations)")) return false;
          if (act) I.state = 2, I.piece = P.chunk_piece[stages[I.t].j];
          return true;
        }
        if (I.state == 2) {  // pieces of the stage's chunk
          const int j = stages[I.t].j;
          while (I.piece < P.chunk_piece[j + 1] && P.piece_owner[I.piece] != q) ++I.piece;
          if (I.piece < P.chunk_piece[j + 1]) {
            const int ns = H.owner_nslots[q], slot = H.owner_slot0[q] + (int)(I.l % ns), use = (int)(I.l / ns);
            if (!wait_ok(w_full[slot], use, use & 1, "issuer (weights)")) return false;
            if (act) w_empty[slot].arrive(), ++I.l, ++I.piece;
            return true;
          }
          if (act) {
            a_empty[I.t % nA].arrive();
            ++I.t;
            if (++I.stage_in_item == (int)item_stages[I.item].size()) {
              acc_full[I.buf].arrive();
              ++I.item, I.stage_in_item = 0, I.state = 0;
            } else {
              I.state = 1;
            }
          }
          return true;
        }
        return false;
      }
      // epilogue
      if (epi.item >= nitems) return false;
      int flip = epi.flip, ph = 0;
      std::vector<int> uses = epi.uses;
      const int buf = acc_buf(epi.item, uses, flip, ph);
      if (!wait_ok(acc_full[buf], ph, ph & 1, "epilogue")) return false;
      if (act) epi.flip = flip, epi.uses = uses, acc_empty[buf].arrive(4), ++epi.item;
      return true;
    };
    const int nact = G + 2 * Q + 1;
    for (int a = 0; a < nact; ++a)
      if (try_actor(a, false)) can.push_back(a);
    if (!err.empty()) break;
    if (can.empty()) {
      bool done = epi.item >= nitems;
      for (int q = 0; q < Q; ++q) done = done && iss[q].item >= nitems && w_next[q] >= own[q].size();
      if (!done) err = "deadlock";
      break;
    }
    try_actor(pick(can), true);
  }
  return err;
}

struct TpResult {
  double err = 0, rz = 0;
  int missing = 0;
};

float bf_at(const unsigned char* blk, int r, int e) {  // element e of row r of a 32-byte-row bf16 block
  const int byte = e * 2;
  uint16_t h;
  std::memcpy(&h, blk + (size_t)r * 32 + ((((byte >> 4) ^ ((r >> 2) & 1)) << 4) | (byte & 15)), 2);
  return bf16_to_f(h);
}
float tf_at(const unsigned char* blk, int r, int e) {
  const int byte = e * 4;
  float w;
  std::memcpy(&w, blk + (size_t)r * 32 + ((((byte >> 4) ^ ((r >> 2) & 1)) << 4) | (byte & 15)), 4);
  return w;
}
float rz_add(float acc, double inc) {  // FP32 add truncated toward zero
  const double x = (double)acc + inc;
  float f = (float)x;
  if (std::fabs((double)f) > std::fabs(x)) f = std::nextafter(f, 0.0f);
  return f;
}

template <typename Entry>
bool tp_check(const char* name, int kind, const TpHost& H, int ncol, int klen, const Entry& entry, bool positive = false,
              TpResult* res = nullptr) {
  const bool split = kind == TC_BF16X3;
  const int kstep = split ? 16 : 8;
  std::mt19937 rng(ncol * 7 + kind);
  std::uniform_real_distribution<double> U(positive ? 0.0 : -1.0, 1.0);
  std::vector<std::vector<float>> A(27, std::vector<float>(klen, 0.f));
  for (auto& r : A)
    for (float& a : r) a = (float)U(rng);
  std::vector<double> ref(ncol, 0), got(ncol, 0), sabs(ncol, 0);
  std::vector<float> gotz(ncol, 0.f);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < klen; ++k)
      for (int n = 0; n < ncol; ++n) {
        const double t = A[d][k] * entry(d, k, n);
        ref[n] += t;
        sabs[n] += std::fabs(t);
      }
  std::vector<int> writer(ncol, -1);
  if (H.w_slots < 1 || H.w_slots > kTpMaxSlots) return fail(name, "ring slots", -1);
  for (int q = 0, s0 = 0; q < kTpIssuers; ++q) {
    if (H.owner_slot0[q] != s0 || H.owner_nslots[q] < 0) return fail(name, "owner rings do not tile the slots", -1);
    s0 += H.owner_nslots[q];
    if (q == kTpIssuers - 1 && s0 != H.w_slots) return fail(name, "owner rings do not tile the slots", -1);
  }
  for (const TpPass& P : H.pass)
    for (int k = 0; k < P.npieces; ++k)
      if (H.owner_nslots[P.piece_owner[k]] < 1) return fail(name, "an owner with pieces has no ring slot", -1);
  if (H.a_stages < 2 || H.a_stages > kTpMaxAStages) return fail(name, "activation stages", -1);
  if (2048 + H.a_stages * kTcAPlaneBytes * (split ? 2 : 1) + H.w_slots * kTpPieceBytes > kTcSmemUsable)
    return fail(name, "shared memory over the budget", -1);
  int mmas = 0;
  for (int ps = 0; ps < (int)H.pass.size(); ++ps) {
    const TpPass& P = H.pass[ps];
    if (P.tmem_cols % 16 || P.tmem_cols * P.nbuf > 512) return fail(name, "more than 512 TMEM columns", ps);
    if (P.chunk_piece[0] != 0 || P.chunk_piece[P.nchunks] != P.npieces) return fail(name, "chunk pieces", ps);
    for (int j = 0; j < P.nchunks; ++j)
      if (P.chunk_piece[j] > P.chunk_piece[j + 1]) return fail(name, "chunk pieces reversed", ps);
    if (P.piece_unit[0] != 0) return fail(name, "piece program", ps);
    for (int g = 0; g < P.ngroups; ++g) {
      if (P.grp_d[g] < 0 || P.grp_d[g] + 16 > P.tmem_cols) return fail(name, "epilogue D outside the set", ps);
      if (P.grp_e[g] >= 0 && P.grp_e[g] + 16 > P.tmem_cols) return fail(name, "epilogue E outside the set", ps);
      if (P.grp_l2[g] >= 0 && P.grp_l2[g] + 16 > P.tmem_cols) return fail(name, "epilogue L2 outside the set", ps);
      for (int c = 0; c < 16 && 16 * g + c < P.ncols; ++c) {
        const int n = P.col0 + 16 * g + c;
        if (n < 0 || n >= ncol) return fail(name, "output column out of range", ps);
        if (writer[n] >= 0) return fail(name, "output column stored by two passes", ps);
        writer[n] = ps;
      }
    }
    // emulate one row: TMEM columns of one set, exact and truncating; every
    // column must be written by one issuer only (fixed summation order)
    std::vector<double> tm(P.tmem_cols, 0.0);
    std::vector<float> tz(P.tmem_cols, 0.f);
    std::vector<int> col_owner(P.tmem_cols, -1);
    auto mma = [&](int tcol, int n, const unsigned char* blk, int row0, int plane, int d, int s, int owner) {
      if (!tp_shape_ok(tcol, n)) return std::string("MMA shape outside the validated forms");
      if (tcol + n > P.tmem_cols) return std::string("MMA writes outside its accumulator set");
      for (int i = 0; i < n; ++i) {
        int& o = col_owner[tcol + i];
        if (o >= 0 && o != owner) return std::string("accumulator column written by two issuers");
        o = owner;
        double acc = 0;
        for (int e = 0; e < kstep; ++e) {
          const int kk = s * kstep + e;
          const float a = kk < klen ? A[d][kk] : 0.f;
          if (split) {
            const float ah = bf16_to_f(bf16_rn(a));
            const float av = plane ? bf16_to_f(bf16_rn(a - ah)) : ah;
            acc += (double)av * bf_at(blk, row0 + i, e);
          } else {
            acc += (double)tf32_trunc(a) * tf_at(blk, row0 + i, e);
          }
        }
        tm[tcol + i] += acc;
        tz[tcol + i] = rz_add(tz[tcol + i], acc);
      }
      ++mmas;
      return std::string();
    };
    for (int xz = 0; xz < 9; ++xz) {
      const int dx = xz % 3 - 1, dz = xz / 3 - 1;
      for (int j = 0; j < P.nchunks; ++j)
        for (int k = P.chunk_piece[j]; k < P.chunk_piece[j + 1]; ++k) {
          const int len = P.piece_len16[k] * 16;
          if (len <= 0 || len > kTpPieceBytes) return fail(name, "piece size", ps);
          if (P.piece_owner[k] < 0 || P.piece_owner[k] >= kTpIssuers) return fail(name, "piece owner", ps);
          const unsigned char* piece = H.W.data() + P.w_base + ((size_t)xz * P.npieces + k) * kTpPieceBytes;
          for (int u = P.piece_unit[k]; u < P.piece_unit[k + 1]; ++u) {
            const uint32_t w = P.unit[u];
            const int b_off = (int)(w & 31u) << 9, ks = (w >> 5) & 3, dy = (w >> 7) & 3, form = (w >> 9) & 3;
            const int tcol = (int)((w >> 11) & 31u) << 4, n = (int)((w >> 16) & 31u) << 4;
            const int tcol2 = (int)((w >> 21) & 31u) << 4;
            if (dy > 2) return fail(name, "bad unit operand", ps);
            if (split != (form != 2)) return fail(name, "unit form against the precision", ps);
            const int rows = form == 2 ? n : 2 * n;
            if (b_off + rows * 32 > len) return fail(name, "unit reads past its piece", ps);
            const int d = (dx + 1) + 3 * dy + 9 * (dz + 1), s = 4 * j + ks, q = P.piece_owner[k];
            std::string e;
            if (form == 0) {  // hi rows then lo rows: hi*hi, lo*hi, hi*lo
              if (e.empty()) e = mma(tcol, n, piece + b_off, 0, 0, d, s, q);
              if (e.empty()) e = mma(tcol, n, piece + b_off, 0, 1, d, s, q);
              if (e.empty()) e = mma(tcol, n, piece + b_off, n, 0, d, s, q);
            } else if (form == 1) {  // hi*[lo reversed; hi] over 2N, then lo*hi
              if (e.empty()) e = mma(tcol, 2 * n, piece + b_off, 0, 0, d, s, q);
              if (e.empty()) e = mma(tcol2, n, piece + b_off, n, 1, d, s, q);
            } else {
              e = mma(tcol, n, piece + b_off, 0, 0, d, s, q);
            }
            if (!e.empty()) return fail(name, e.c_str(), ps);
          }
        }
    }
    for (int g = 0; g < P.ngroups; ++g)
      for (int c = 0; c < 16 && 16 * g + c < P.ncols; ++c) {
        const int n = P.col0 + 16 * g + c;
        double v = tm[P.grp_d[g] + c];
        float vz = tz[P.grp_d[g] + c];
        if (P.grp_e[g] >= 0) v += tm[P.grp_e[g] + 15 - c], vz += tz[P.grp_e[g] + 15 - c];
        if (P.grp_l2[g] >= 0) v += tm[P.grp_l2[g] + c], vz += tz[P.grp_l2[g] + c];
        got[n] = v;
        gotz[n] = vz;
      }
  }
  for (unsigned seed = 1; seed <= 20; ++seed) {
    const std::string e = simulate_protocol(H, kind, 3 * (int)H.pass.size(), seed);
    if (!e.empty()) return fail(name, ("barrier protocol: " + e).c_str(), -1);
  }
  TpResult R;
  for (int n = 0; n < ncol; ++n) {
    R.missing += writer[n] < 0;
    if (sabs[n] > 0) {
      R.err = std::max(R.err, std::fabs(got[n] - ref[n]) / sabs[n]);
      R.rz = std::max(R.rz, std::fabs((double)gotz[n] - ref[n]) / sabs[n]);
    }
  }
  if (res) *res = R;
  const double tol = split ? 2e-5 : 1e-3;
  size_t pieces = 0;
  int maxset = 0;
  for (const TpPass& P : H.pass) pieces += P.npieces, maxset = std::max(maxset, P.tmem_cols * P.nbuf);
  std::printf("%-28s %-6s passes %d mmas/tile %5d pieces/column %3zu tmem %3d weights %6.2f MB uncovered %d "
              "err/sum|terms| %.2e rz %.2e\n",
              name, split ? "bf16x3" : "tf32", (int)H.pass.size(), mmas, pieces, maxset, H.W.size() / 1e6,
              R.missing, R.err, R.rz);
  if (R.missing) return fail(name, "output columns never written", -1);
  if (!(R.err <= tol)) return fail(name, "result differs from the direct contraction", -1);
  return true;
}

bool tp_m2l_case(int kind, int p, int mult_order, int local_order, bool harm, bool& built) {
  MultiIndex mi;
  mi.init(p);
  if (mult_order >= 0) mi.mo = mult_order;
  if (local_order >= 0) mi.lo = local_order;
  TaylorTable tt;
  tt.build(mi);
  TpHost H;
  char name[64];
  std::snprintf(name, sizeof name, "m2l p=%d mo=%d lo=%d%s", p, mi.mo, mi.lo, harm ? " harmonic" : "");
  built = build_tp_m2l(mi, tt, kind, H, harm);
  if (!built) {
    std::printf("%-28s %-6s span schedule (no prefix schedule)\n", name, kind == TC_BF16X3 ? "bf16x3" : "tf32");
    return true;
  }
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  return tp_check(name, kind, H, 8 * nk, 8 * nk, [&](int d, int k, int n) {
    return harm ? m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8) : m2l_entry(mi, tt, d, k, n);
  });
}

bool tp_m2p_case(int kind, int p, int b, int mult_order, bool harm, bool& built, int comps = 1) {
  MultiIndex mi, mi1;
  mi.init(p);
  mi1.init(p + 1);
  if (mult_order >= 0) mi.mo = mult_order;
  M2pTable tab;
  tab.build(comps > 1 ? mi1 : mi, b);
  TpHost H;
  char name[64];
  std::snprintf(name, sizeof name, "m2p p=%d mo=%d b=%d%s%s", p, mi.mo, b, harm ? " harmonic" : "",
                comps > 1 ? " force" : "");
  built = build_tp_m2p(mi, tab, kind, H, harm, comps);
  if (!built) {
    std::printf("%-28s %-6s span schedule (no prefix schedule)\n", name, kind == TC_BF16X3 ? "bf16x3" : "tf32");
    return true;
  }
  const std::vector<int> red = harmonic_components(mi);
  const int nk = harm ? (int)red.size() : mi.nc;
  return tp_check(name, kind, H, 8 * comps * b * b * b, 8 * nk, [&](int d, int k, int n) {
    return harm ? m2p_entry(mi, tab, d, red[k / 8] * 8 + k % 8, n, comps) : m2p_entry(mi, tab, d, k, n, comps);
  });
}

bool tp_near_case(int b, int comps, bool& built) {
  TpHost H;
  char name[64];
  std::snprintf(name, sizeof name, "near b=%d columns=%d", b, comps);
  built = build_tp_near(b, comps, TC_BF16X3, H);
  if (!built) {
    std::printf("%-28s %-6s span schedule (no prefix schedule)\n", name, "bf16x3");
    return true;
  }
  return tp_check(name, TC_BF16X3, H, comps * b * b * b, b * b * b, [b](int d, int k, int n) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    return near_entry(b, D, k, n);
  });
}

// Every configuration the span schedule covers; `built` counts the ones with
// a prefix schedule.
int prefix_check(int& built_count) {
  bool ok = true, built = false;
  built_count = 0;
  for (int kind : {TC_BF16X3, TC_TF32})
    for (int p : {2, 4, 6, 8})
      for (bool harm : {false, true}) ok &= tp_m2l_case(kind, p, -1, -1, harm, built), built_count += built;
  for (int p : {3, 4, 6})
    for (bool harm : {false, true}) {
      ok &= tp_m2l_case(TC_BF16X3, p, p - 1, -1, harm, built), built_count += built;
      ok &= tp_m2l_case(TC_BF16X3, p, -1, p - 1, harm, built), built_count += built;
      ok &= tp_m2p_case(TC_BF16X3, p, 2, p - 1, harm, built), built_count += built;
    }
  for (int kind : {TC_BF16X3, TC_TF32})
    for (int p : {4, 6})
      for (int b : {2, 4})
        for (bool harm : {false, true}) ok &= tp_m2p_case(kind, p, b, -1, harm, built), built_count += built;
  for (int b : {2, 4, 8})
    for (int comps : {1, 4}) ok &= tp_near_case(b, comps, built), built_count += built;
  for (int kind : {TC_BF16X3, TC_TF32})  // the final-stage M2P with the force's gradient columns
    for (int b : {2, 4})
      for (bool harm : {false, true}) ok &= tp_m2p_case(kind, 6, b, -1, harm, built, 4), built_count += built;
  return ok ? 0 : 1;
}

// The span schedule (build_tc) under the same truncating accumulation: one
// FP32 add per MMA (K step and product) into its span's accumulator.
double span_rz_error(const TcHost& H, int kind, int ncol, int klen, const std::function<double(int, int, int)>& entry,
                     bool positive) {
  const int chunk = kind == TC_BF16X3 ? 64 : 32, kstep = chunk / 4, esz = kind == TC_BF16X3 ? 2 : 4;
  std::mt19937 rng(ncol * 7 + kind);
  std::uniform_real_distribution<double> U(positive ? 0.0 : -1.0, 1.0);
  std::vector<std::vector<float>> A(27, std::vector<float>(klen, 0.f));
  for (auto& r : A)
    for (float& a : r) a = (float)U(rng);
  std::vector<double> ref(ncol, 0), sabs(ncol, 0);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < klen; ++k)
      for (int n = 0; n < ncol; ++n) {
        const double t = A[d][k] * entry(d, k, n);
        ref[n] += t;
        sabs[n] += std::fabs(t);
      }
  std::vector<double> got(ncol, 0);
  for (int ps = 0; ps < H.npass; ++ps) {
    const TcPass& P = H.pass[ps];
    std::vector<float> tz(512, 0.f);
    for (int xz = 0; xz < 9; ++xz)
      for (int j = 0; j < P.nchunks; ++j)
        for (int dy = 0; dy < 3; ++dy) {
          const int d = (xz % 3) + 3 * dy + 9 * (xz / 3);
          for (int si = P.span_idx[j][0]; si < P.span_idx[j][kTcIssuers]; ++si) {
            const TcSpan& S = P.span[si];
            const unsigned char* tile = H.W.data() + P.w_base + (size_t)d * P.bytes_per_d + S.w_off;
            for (int r = 0; r < S.n; ++r)
              for (int ks = 0; ks < S.ksteps; ++ks) {
                const int nprod = kind == TC_BF16X3 && S.prod == 0 ? 3 : 1;
                for (int pr = 0; pr < nprod; ++pr) {
                  double acc = 0;
                  for (int e = ks * kstep; e < (ks + 1) * kstep; ++e) {
                    const int k = j * chunk + e;
                    const float a = k < klen ? A[d][k] : 0.f;
                    const int byte = e * esz;
                    const size_t off = (size_t)r * 128 + (size_t)((((byte >> 4) ^ (r & 7)) << 4) | (byte & 15));
                    if (kind == TC_BF16X3) {
                      const float ah = bf16_to_f(bf16_rn(a)), al = bf16_to_f(bf16_rn(a - ah));
                      uint16_t w1, wl;
                      std::memcpy(&w1, tile + off, 2);
                      if (S.prod == 0) {
                        std::memcpy(&wl, tile + (size_t)S.n * 128 + off, 2);
                        acc += pr == 0 ? (double)ah * bf16_to_f(w1) : pr == 1 ? (double)ah * bf16_to_f(wl)
                                                                             : (double)al * bf16_to_f(w1);
                      } else {
                        acc += (double)(S.prod == 3 ? al : ah) * bf16_to_f(w1);
                      }
                    } else {
                      float w;
                      std::memcpy(&w, tile + off, 4);
                      acc += (double)tf32_trunc(a) * w;
                    }
                  }
                  tz[S.tmem_col + r] = rz_add(tz[S.tmem_col + r], acc);
                }
              }
          }
        }
    for (int g = 0; g < P.ng; ++g)
      for (int c = 0; c < P.out_ncols[g]; ++c) {
        double v = tz[P.out_tmem[g] + c];
        if (P.out_tmem2[g] >= 0) v += tz[P.out_tmem2[g] + c];
        if (P.out_tmem3[g] >= 0) v += tz[P.out_tmem3[g] + c];
        if (P.out_tmem4[g] >= 0) v += tz[P.out_tmem4[g] + c];
        got[P.out_col0[g] + c] = v;
      }
  }
  double err = 0;
  for (int n = 0; n < ncol; ++n)
    if (sabs[n] > 0) err = std::max(err, std::fabs(got[n] - ref[n]) / sabs[n]);
  return err;
}

// Accumulator rounding of the span and prefix schedules on same-signed
// activations (order 6 harmonic M2L, the near field of leaf 4), for the record.
int rounding_report() {
  MultiIndex mi;
  mi.init(6);
  TaylorTable tt;
  tt.build(mi);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = (int)red.size();
  auto entry = [&](int d, int k, int n) { return m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8); };
  TpHost H;
  TpResult R;
  if (!build_tp_m2l(mi, tt, TC_BF16X3, H, true)) return 1;
  if (!tp_check("m2l p=6 harmonic, A >= 0", TC_BF16X3, H, 8 * nk, 8 * nk, entry, true, &R)) return 1;
  TcHost Hs;
  if (!build_tc(mi, tt, TC_BF16X3, Hs, true)) return 1;
  std::printf("%-28s span schedule rz %.2e\n", "m2l p=6 harmonic, A >= 0",
              span_rz_error(Hs, TC_BF16X3, 8 * nk, 8 * nk, entry, true));
  TpHost Hn;
  TpResult Rn;
  if (!build_tp_near(4, 1, TC_BF16X3, Hn)) return 1;
  if (!tp_check("near b=4, A >= 0", TC_BF16X3, Hn, 64, 64, [](int d, int k, int n) {
        const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
        return near_entry(4, D, k, n);
      }, true, &Rn))
    return 1;
  TcHost Hns;
  if (!build_tc_near(4, 1, TC_BF16X3, Hns)) return 1;
  std::printf("%-28s span schedule rz %.2e\n", "near b=4, A >= 0",
              span_rz_error(Hns, TC_BF16X3, 64, 64, [](int d, int k, int n) {
                const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
                return near_entry(4, D, k, n);
              }, true));
  return 0;
}

// Planted mistakes in a built prefix schedule (order 6, harmonic, bf16x3),
// each of which the check must catch.  Returns the number that were not.
int planted_prefix_mistakes() {
  MultiIndex mi;
  mi.init(6);
  TaylorTable tt;
  tt.build(mi);
  const std::vector<int> red = harmonic_components(mi);
  const int nk = (int)red.size();
  auto entry = [&](int d, int k, int n) { return m2l_entry(mi, tt, d, red[k / 8] * 8 + k % 8, red[n / 8] * 8 + n % 8); };
  int missed = 0;
  auto plant = [&](const char* what, auto corrupt) {
    TpHost H;
    if (!build_tp_m2l(mi, tt, TC_BF16X3, H, true) || !corrupt(H)) {
      std::printf("planted mistake could not be placed: %s\n", what);
      ++missed;
      return;
    }
    if (tp_check(what, TC_BF16X3, H, 8 * nk, 8 * nk, entry)) {
      std::printf("planted mistake NOT caught: %s\n", what);
      ++missed;
    }
  };
  auto first_form = [](const TpPass& P, int form) {
    for (int u = 0; u < P.piece_unit[P.npieces]; ++u)
      if ((int)((P.unit[u] >> 9) & 3u) == form) return u;
    return -1;
  };
  {  // the protocol replay must reject two owners taking turns on one ring slot
    TpHost H;
    if (!build_tp_m2l(mi, tt, TC_BF16X3, H, true)) {
      ++missed;
    } else {
      int q0 = -1, q1 = -1;  // two owners with pieces: the second's ring moved onto the first's
      for (int q = 0; q < kTpIssuers; ++q)
        if (H.owner_nslots[q] > 0) (q0 < 0 ? q0 : q1) = q0 < 0 ? q : (q1 < 0 ? q : q1);
      int bad = 0;
      if (q0 >= 0 && q1 >= 0) {
        H.owner_slot0[q1] = H.owner_slot0[q0];
        H.owner_nslots[q1] = H.owner_nslots[q0];
        for (unsigned seed = 1; seed <= 40; ++seed) bad += !simulate_protocol(H, TC_BF16X3, 3, seed).empty();
      }
      std::printf("two owners on one ring: %d of 40 replays fail the protocol check\n", bad);
      if (bad == 0) {
        std::printf("planted mistake NOT caught: two owners on one ring\n");
        ++missed;
      }
    }
  }
  plant("zeroed weight block", [](TpHost& H) {  // the first block of the first column (dx = dz = -1)
    const TpPass& P = H.pass[0];
    std::fill_n(H.W.begin() + P.w_base, 4096, (unsigned char)0);
    return true;
  });
  plant("block row read unswizzled", [](TpHost& H) {  // row 5: its 16-byte halves trade places
    const TpPass& P = H.pass[0];
    unsigned char* row = H.W.data() + P.w_base + 5 * 32;
    std::swap_ranges(row, row + 16, row + 16);
    return true;
  });
  plant("unit into the wrong accumulator columns", [&](TpHost& H) {
    TpPass& P = H.pass[0];
    const int u = first_form(P, 0);
    if (u < 0) return false;
    P.unit[u] += 1u << 11;  // TMEM column + 16
    return true;
  });
  plant("unit on the wrong dy window", [](TpHost& H) {
    TpPass& P = H.pass[0];
    P.unit[0] = (P.unit[0] & ~(3u << 7)) | (((((P.unit[0] >> 7) & 3u) + 1) % 3) << 7);
    return true;
  });
  plant("unit on the wrong K step of its chunk", [](TpHost& H) {
    TpPass& P = H.pass[0];
    P.unit[0] ^= 1u << 5;
    return true;
  });
  plant("fused MMA one group off in E", [&](TpHost& H) {  // its reversed columns land one group late
    TpPass& P = H.pass[0];
    for (int u = 0; u < P.piece_unit[P.npieces]; ++u)
      if (((P.unit[u] >> 9) & 3u) == 1 && ((P.unit[u] >> 16) & 31u) <= 2) {  // N <= 32: room to shift
        P.unit[u] += 1u << 11;
        return true;
      }
    return false;
  });
  plant("epilogue reads E unreversed", [](TpHost& H) {
    TpPass& P = H.pass[0];
    if (P.grp_e[0] < 0 || P.ngroups < 2 || P.grp_e[1] < 0) return false;
    std::swap(P.grp_e[0], P.grp_e[1]);
    return true;
  });
  plant("epilogue drops the L2 region", [](TpHost& H) {
    TpPass& P = H.pass[0];
    if (P.grp_l2[0] < 0) return false;
    P.grp_l2[0] = -1;
    return true;
  });
  plant("piece cut one unit early", [](TpHost& H) {
    TpPass& P = H.pass[0];
    if (P.npieces < 2 || P.piece_unit[1] - P.piece_unit[0] < 2) return false;
    P.piece_unit[1] -= 1;
    return true;
  });
  plant("piece read by a second issuer", [](TpHost& H) {  // its columns then have two writers
    TpPass& P = H.pass[0];
    for (int k = 1; k < P.npieces; ++k)
      if (P.piece_owner[k] != P.piece_owner[0]) {
        for (int k2 = 0; k2 < P.npieces; ++k2)  // a piece of the first piece's owner moves to another issuer
          if (k2 != 0 && P.piece_owner[k2] == P.piece_owner[0]) {
            P.piece_owner[k2] = P.piece_owner[k];
            return true;
          }
      }
    return false;
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

// Final-stage M2P weights with the analytic force's three gradient columns
// [27][8 nc][8 x 4 b^3] (neighbour parent, alpha * 8 + source child,
// target child * 4 b^3 + component * b^3 + cell), Taylor table to order p + 1.
bool dump_m2p_grad(const std::string& dir, int p, int b) {
  MultiIndex mi, mi1;
  mi.init(p);
  mi1.init(p + 1);
  M2pTable tab;
  tab.build(mi1, b);
  const int K = 8 * mi.nc, N = 8 * 4 * b * b * b;
  std::vector<double> W((size_t)27 * K * N);
  for (int d = 0; d < 27; ++d)
    for (int k = 0; k < K; ++k)
      for (int n = 0; n < N; ++n) W[((size_t)d * K + k) * N + n] = m2p_entry(mi, tab, d, k, n, 4);
  char name[64];
  std::snprintf(name, sizeof name, "/m2pg_p%d_b%d.bin", p, b);
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

// The dedicated leaf-4 near-field kernel (k_near_tc.cu): its weight image
// decoded with the 128-byte swizzle the MMA reads (row n, 16-byte chunk
// (2k / 16) xor (n mod 8)), hi + lo against near_entry, and its products
// (hi*lo + lo*hi + hi*hi over the 27 neighbours, lo*lo dropped) emulated on
// random densities against the FP64 contraction.
int near4_check() {
  std::vector<unsigned char> W4;
  near4_weights(W4);
  if (W4.size() != (size_t)27 * kNtPieceBytes) return std::printf("near4: image size %zu\n", W4.size()), 1;
  auto rd = [&](int d, int plane, int n, int k) {
    const size_t o = (size_t)d * kNtPieceBytes + (size_t)plane * (kNtPieceBytes / 2) + (size_t)n * 128 +
                     (size_t)((((2 * k) >> 4) ^ (n & 7)) << 4) + (size_t)((2 * k) & 15);
    uint16_t h;
    std::memcpy(&h, W4.data() + o, 2);
    return (double)bf16_to_f(h);
  };
  double split = 0.0;
  for (int d = 0; d < 27; ++d) {
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    for (int n = 0; n < 64; ++n)
      for (int k = 0; k < 64; ++k) {
        const double w = near_entry(4, D, k, n);
        split = std::max(split, std::fabs(rd(d, 0, n, k) + rd(d, 1, n, k) - w) / std::fabs(w));
      }
  }
  std::mt19937 rng(4);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double worst = 0.0;
  for (int trial = 0; trial < 4; ++trial) {
    std::vector<double> A(27 * 64);
    for (double& a : A) a = U(rng);
    for (int n = 0; n < 64; ++n) {
      double exact = 0.0, mag = 0.0, emul = 0.0;
      for (int d = 0; d < 27; ++d) {
        const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
        for (int k = 0; k < 64; ++k) {
          const double a = A[d * 64 + k], w = near_entry(4, D, k, n);
          const double ah = bf16_to_f(bf16_rn((float)a)), al = bf16_to_f(bf16_rn((float)(a - ah)));
          exact += a * w;
          mag += std::fabs(a * w);
          emul += ah * rd(d, 1, n, k) + al * rd(d, 0, n, k) + ah * rd(d, 0, n, k);
        }
      }
      worst = std::max(worst, std::fabs(emul - exact) / mag);
    }
  }
  std::printf("near4: hi + lo vs weight %.2e, products vs FP64 %.2e of sum |terms|\n", split, worst);
  return (split <= 1.0 / 65536.0 && worst <= 1e-5) ? 0 : 1;
}

// The dedicated near-field kernel's barrier protocol (k_near_tc.cu) replayed
// on the CPU with the kernel's stage, group and set arithmetic: the
// activation producer (boxes in (item, column, tile) order over a 3-stage
// ring), the weight producer (one 3-piece group per column, two buffers), the
// two issuers (tiles 0-1 / 2-3; the accumulator set of each column segment,
// the group, their boxes; one commit per box, group and segment), the 16
// epilogue warps (one hand-off per segment).  Work items hold 4 tiles, the
// last one possibly fewer.  Each run picks actors at random with skewed
// speeds; every wait must agree with the phase the protocol means and every
// actor must finish.
std::string simulate_near4(int nitems, int last_tiles, unsigned seed, int plant = 0) {
  constexpr int nA = 3;
  std::vector<SimBar> a_full(nA), a_empty(nA), w_full(2), w_empty(2), acc_full(2), acc_empty(2);
  for (auto& b : w_empty) b.expected = 2;
  for (auto& b : acc_full) b.expected = 2;
  for (auto& b : acc_empty) b.expected = 16;
  auto tiles_of = [&](int item) { return item == nitems - 1 ? last_tiles : 4; };
  std::string err;
  auto wait_ok = [&](const SimBar& b, int phase_index, uint32_t parity, const char* who) {
    const bool intended = b.done > phase_index, hardware = b.hw(parity);
    if (intended != hardware && err.empty())
      err = std::string(who) + ": a parity wait that does not match its phase (" +
            (hardware ? "passes early" : "would hang") + ")";
    return intended && hardware;
  };
  // A producer: box sequence (item, g, t)
  struct Box { int item, g, t; };
  std::vector<Box> boxes;
  for (int it = 0; it < nitems; ++it)
    for (int g = 0; g < 9; ++g)
      for (int t = 0; t < tiles_of(it); ++t) boxes.push_back({it, g, t});
  size_t a_next = 0;
  int w_next = 0;  // next group gi
  const int ngroups = 9 * nitems;
  struct Iss { int gi = 0, state = 0, t = 0; size_t ai = 0; };
  Iss iss[2];
  int epi[16] = {};
  std::mt19937 rng(seed);
  std::vector<double> speed(2 + 2 + 16);
  for (double& v : speed) v = std::pow(10.0, (double)(rng() % 3));
  for (int step = 0; step < 10000000 && err.empty(); ++step) {
    auto try_actor = [&](int a, bool act) -> bool {
      if (a == 0) {  // activation producer
        if (a_next >= boxes.size()) return false;
        const int sa = (int)(a_next % nA), use = (int)(a_next / nA);
        if (!wait_ok(a_empty[sa], use - 1, (uint32_t)((use & 1) ^ 1), "activation producer")) return false;
        if (act) a_full[sa].arrive(), ++a_next;
        return true;
      }
      if (a == 1) {  // weight producer
        if (w_next >= ngroups) return false;
        const int wb = w_next & 1, use = w_next >> 1;
        if (!wait_ok(w_empty[wb], use - 1, (uint32_t)((use & 1) ^ 1), "weight producer")) return false;
        if (act) w_full[wb].arrive(), ++w_next;
        return true;
      }
      if (a < 4) {  // issuer q
        const int q = a - 2;
        Iss& I = iss[q];
        if (I.gi >= ngroups) return false;
        const int item = I.gi / 9, set = I.gi & 1, use = I.gi >> 1;
        if (I.state == 0) {
          if (!wait_ok(acc_empty[set], use - 1, (uint32_t)((use & 1) ^ 1), "issuer (accumulators)")) return false;
          if (act) I.state = 1;
          return true;
        }
        if (I.state == 1) {
          if (!wait_ok(w_full[I.gi & 1], I.gi >> 1, (uint32_t)((I.gi >> 1) & 1), "issuer (weights)")) return false;
          if (act) I.state = 2, I.t = 0;
          return true;
        }
        // state 2: the item's tiles in order (mine: wait and commit the box; every valid tile advances ai)
        if (I.t < tiles_of(item)) {
          if ((I.t >> 1) == q) {
            const int sa = (int)(I.ai % nA), u = (int)(I.ai / nA);
            if (!wait_ok(a_full[sa], u, (uint32_t)((u + (plant == 1)) & 1), "issuer (activations)")) return false;
            if (act) a_empty[sa].arrive();
          }
          if (act) ++I.ai, ++I.t;
          return true;
        }
        if (act) w_empty[I.gi & 1].arrive(), acc_full[set].arrive(), ++I.gi, I.state = 0;
        return true;
      }
      const int e = a - 4;  // epilogue warp
      if (epi[e] >= ngroups) return false;
      const int set = epi[e] & 1, use = epi[e] >> 1;
      if (!wait_ok(acc_full[set], use, (uint32_t)(use & 1), "epilogue")) return false;
      if (act) {
        if (!(plant == 2 && e == 0 && epi[e] % 9 != 8)) acc_empty[set].arrive();  // planted: one hand-off per item
        ++epi[e];
      }
      return true;
    };
    std::vector<int> can;
    for (int a = 0; a < 20; ++a)
      if (try_actor(a, false)) can.push_back(a);
    if (!err.empty()) break;
    if (can.empty()) {
      bool done = a_next >= boxes.size() && w_next >= ngroups && iss[0].gi >= ngroups && iss[1].gi >= ngroups;
      for (int e = 0; e < 16; ++e) done = done && epi[e] >= ngroups;
      if (!done) err = "deadlock";
      break;
    }
    double tot = 0;
    for (int a : can) tot += speed[a];
    double r = tot * (rng() / (double)rng.max());
    int pickd = can.back();
    for (int a : can)
      if ((r -= speed[a]) <= 0) {
        pickd = a;
        break;
      }
    try_actor(pickd, true);
  }
  return err;
}

int near4_protocol_check() {
  int bad = 0, runs = 0;
  for (int nitems : {1, 2, 3, 7})
    for (int last : {1, 2, 3, 4})
      for (unsigned seed = 1; seed <= 25; ++seed, ++runs) {
        const std::string e = simulate_near4(nitems, last, seed * 7919u + nitems * 31u + last);
        if (!e.empty()) {
          if (bad < 5) std::printf("near4 protocol: %d items, last %d tiles, seed %u: %s\n", nitems, last, seed, e.c_str());
          ++bad;
        }
      }
  std::printf("near4 protocol: %d of %d randomised replays clean\n", runs - bad, runs);
  // planted mistakes must be caught: a wrong parity on the issuers' activation
  // wait; one epilogue warp handing back its accumulators once per item
  for (int plant : {1, 2}) {
    int caught = 0;
    for (unsigned seed = 1; seed <= 10; ++seed) caught += !simulate_near4(3, 2, seed, plant).empty();
    std::printf("near4 protocol: planted mistake %d caught in %d of 10 replays\n", plant, caught);
    bad += caught == 0;
  }
  return bad ? 1 : 0;
}

// The CUDA-core M2L kernels skip the centre neighbour's weight block
// (NbrGemm::skip_center): it must be all zero, and no other block may be.
// A parent's children are each other's near neighbours (Chebyshev distance
// <= 1), so none is in another's interaction list (Sec. 2.2).
int centre_check() {
  int bad = 0;
  for (int p : {2, 4, 6, 8})
    for (bool harm : {false, true})
      for (int lim = 0; lim < 3; ++lim) {  // symmetric orders; mult_order = p - 1; its transpose
      MultiIndex mi;
      mi.init(p);
      if (lim == 1) mi.mo = p - 1;
      if (lim == 2) mi.lo = p - 1;
      TaylorTable tt;
      tt.build(mi);
      std::vector<double> W;
      std::vector<int> tk;
      std::vector<long long> tw;
      m2l_weights<double>(mi, tt, W, tk, tw, true, harm);
      long long centre = 0, zero_blocks = 0;
      for (size_t t = 0; t < tk.size(); ++t)
        for (int d = 0; d < 27; ++d) {
          const double* blk = W.data() + tw[t] + (long long)d * tk[t] * kNTile;
          long long nz = 0;
          for (long long i = 0; i < (long long)tk[t] * kNTile; ++i) nz += blk[i] != 0.0;
          if (d == 13) centre += nz;
          else if (nz == 0 && t == 0) ++zero_blocks;
        }
      std::printf("centre: p=%d harm=%d limits %d: nonzero centre weights %lld, other zero blocks of tile 0 %lld\n",
                  p, harm, lim, centre, zero_blocks);
      bad += centre != 0 || zero_blocks != 0;
      }
  return bad ? 1 : 0;
}

// ---------------------------------------------------------------------------
// The fused batch's work tables.  Plans are built layout-only (placeholder
// device addresses, no device work) and the library's build_fused writes the
// steps and the item tables of one batched solve; the replay here checks:
//  * the launches come in the order of the method's steps (P2M, M2M, M2L and
//    near field, L2L, leaf evaluation, force), every field's M2M from its
//    leaf level up to level 3 one level per launch, its L2L from level 2 down
//    (the leaf level's in the leaf kernel where the plan fuses it), one
//    absolute level per L2L launch, and every M2L level and near field of
//    every field in exactly one contraction launch;
//  * each launch's block ranges tile [0, blocks) with no gap or overlap, and
//    every launch block maps (multi.cuh's lookup, as the kernels run it) to
//    one block of one item's own grid;
//  * each contraction item's tile form and grid: the tiny form for grids of
//    at most 64 rows, the 6-row z-run where it pads z less than the 8-row run
//    (FP32), and the z-run tiles (8 x 4 x RZ rows, one per column tile) cover
//    every row of the item's grid once;
//  * the leaf items carry the leaf-level L2L exactly where the plan fuses it,
//    and every item reads and writes its own field's buffers.
namespace batchcheck {

constexpr int kBx = 8, kBy = 4;  // z-run tile extent in x and y (k_gemm_zrun.cu)

struct Case {
  std::vector<fmm_plan_t> plans;
  std::vector<const void*> rho;
  std::vector<void*> phi, acc;
  bool f64 = false, accel = true;
  ~Case() {
    for (fmm_plan_t P : plans) delete P;
  }
};

fmm_plan_t dry_plan(const int d3[3], int order, int leaf, bool f64, int index) {
  fmm_opts o;
  fmm_default_opts(&o);
  o.precision = f64 ? FMM_FP64 : FMM_FP32;
  o.accel = 1;
  fmm_plan_t P = new fmm_plan_s();
  // placeholder addresses: one 1 TB range per field, never dereferenced
  P->static_base = reinterpret_cast<unsigned char*>((uintptr_t)(index + 1) << 40);
  P->static_cap = (size_t)1 << 39;
  P->static_keep_tables = true;
  P->dry = true;
  if (plan_init(P, d3, 1.0 / d3[0], 1.0, order, leaf, o, nullptr, 0) != FMM_OK) {
    std::printf("batch: plan %dx%dx%d failed: %s\n", d3[0], d3[1], d3[2], fmm_last_error());
    delete P;
    return nullptr;
  }
  return P;
}

template <typename A>
const A* items(const std::vector<unsigned char>& tab, const MultiStep& st) {
  return reinterpret_cast<const A*>(tab.data() + st.args_off);
}
const MultiGrid* grids(const std::vector<unsigned char>& tab, const MultiStep& st) {
  return reinterpret_cast<const MultiGrid*>(tab.data() + st.grids_off);
}

// The z-run length of a contraction tile form (the kernels' template RZ).
int zrun_len(int shape, bool f64) { return shape == 5 ? (f64 ? 3 : 6) : (f64 ? 4 : 8); }

// Every check above; the first failure is reported in *why.
bool check(const Case& c, const std::vector<MultiStep>& steps, const std::vector<unsigned char>& tab,
           std::string* why) {
  auto fail = [&](const std::string& m) {
    *why = m;
    return false;
  };
  const int nf = (int)c.plans.size();
  // --- order of the launches and block ranges ---
  for (size_t k = 0; k < steps.size(); ++k) {
    const MultiStep& st = steps[k];
    if (k && st.kind < steps[k - 1].kind) return fail("launch " + std::to_string(k) + " out of step order");
    if (st.n <= 0 || st.blocks <= 0 || st.blocks > 0x7fffffffLL) return fail("launch " + std::to_string(k) + " size");
    if (st.args_off % 16 || st.grids_off % 16 || st.grids_off + st.n * sizeof(MultiGrid) > tab.size())
      return fail("launch " + std::to_string(k) + " table placement");
    const MultiGrid* g = grids(tab, st);
    long long next = 0;
    for (int i = 0; i < st.n; ++i) {
      const long long nb = (long long)g[i].gx * g[i].gy * g[i].gz;
      if (g[i].start != next || nb <= 0) return fail("launch " + std::to_string(k) + " block ranges");
      next += nb;
    }
    if (next != st.blocks) return fail("launch " + std::to_string(k) + " block total");
    std::vector<long long> seen(st.n, 0);
    for (long long b = 0; b < st.blocks; ++b) {
      const int i = multi_item_at(g, st.n, b);
      const long long nb = (long long)g[i].gx * g[i].gy * g[i].gz;
      const VBlock v = multi_vblock_at(g[i], b);
      if (b < g[i].start || b >= g[i].start + nb || v.x >= v.gx || v.y >= v.gy || v.z >= v.gz ||
          ((long long)v.z * v.gy + v.y) * v.gx + v.x != b - g[i].start)
        return fail("launch " + std::to_string(k) + " block " + std::to_string(b) + " maps outside its item");
      ++seen[i];
    }
    for (int i = 0; i < st.n; ++i)
      if (seen[i] != (long long)g[i].gx * g[i].gy * g[i].gz) return fail("launch " + std::to_string(k) + " coverage");
  }
  // --- per field: which launch holds each of its steps ---
  std::vector<int> p2m(nf, 0), leaf(nf, 0), fd(nf, 0), m2m_next(nf), l2l_next(nf, 1);
  std::vector<std::vector<int>> gemm(nf);
  for (int f = 0; f < nf; ++f) {
    m2m_next[f] = c.plans[f]->L;
    gemm[f].assign(c.plans[f]->L + 2, 0);  // levels 2 .. L, then the near field at L + 1
  }
  auto field_of = [&](const void* ptr) {
    for (int f = 0; f < nf; ++f) {
      const unsigned char* a = c.plans[f]->arena;
      const unsigned char* q = static_cast<const unsigned char*>(ptr);
      if (q >= a && q < a + c.plans[f]->arena_bytes) return f;
    }
    return -1;
  };
  int l2l_level_prev = 1;
  for (size_t k = 0; k < steps.size(); ++k) {
    const MultiStep& st = steps[k];
    const MultiGrid* g = grids(tab, st);
    const std::string at = "launch " + std::to_string(k);
    if (st.kind == MK_P2M) {
      const P2mArgs* a = items<P2mArgs>(tab, st);
      for (int i = 0; i < st.n; ++i) {
        const int f = field_of(a[i].Mleaf);
        if (f < 0 || a[i].Mleaf != c.plans[f]->M(c.plans[f]->L) || a[i].rho != c.rho[f]) return fail(at + ": P2M item");
        ++p2m[f];
      }
    } else if (st.kind == MK_M2M) {
      const M2mArgs* a = items<M2mArgs>(tab, st);
      for (int i = 0; i < st.n; ++i) {
        const int f = field_of(a[i].Mc);
        if (f < 0) return fail(at + ": M2M item of no field");
        const fmm_plan_t P = c.plans[f];
        const int l = m2m_next[f];
        if (l < 3 || a[i].Mc != P->M(l) || a[i].Mp != P->M(l - 1)) return fail(at + ": M2M out of level order");
        --m2m_next[f];
      }
    } else if (st.kind == MK_GEMM) {
      const NbrGemm* a = items<NbrGemm>(tab, st);
      for (int i = 0; i < st.n; ++i) {
        const NbrGemm& x = a[i];
        const int f = field_of(x.C);
        if (f < 0) return fail(at + ": contraction of no field");
        const fmm_plan_t P = c.plans[f];
        int which = -1;
        std::vector<int> tk;
        for (int l = 2; l <= P->L; ++l)
          if (x.C == m2l_gemm(P, l).C) which = l, tk = P->h_m2l_tile_k;
        if (x.C == near_gemm(P).C) which = P->L + 1, tk = P->h_near_tile_k;
        if (which < 0) return fail(at + ": contraction writes no level");
        ++gemm[f][which];
        const NbrGemm ref = which <= P->L ? m2l_gemm(P, which) : near_gemm(P);
        if (x.A != ref.A || x.W != ref.W || x.ntiles != ref.ntiles || x.n_cols != ref.n_cols ||
            x.row_len != ref.row_len || x.skip_center != ref.skip_center || x.grid[0] != ref.grid[0] ||
            x.grid[1] != ref.grid[1] || x.grid[2] != ref.grid[2])
          return fail(at + ": contraction differs from the plan's");
        if (x.dsplit != 1 || x.partial) return fail(at + ": neighbour split inside the batch");
        if (x.shape != st.shape) return fail(at + ": item of another tile form");
        const long long rows = (long long)x.grid[0] * x.grid[1] * x.grid[2];
        if (st.shape == 4) {
          if (!nbr_gemm_tiny_fits(x) || rows > 64 || g[i].gx != (unsigned)x.ntiles || g[i].gy != 1 || g[i].gz != 1)
            return fail(at + ": tiny-grid item");
        } else if (st.shape == 1 || st.shape == 5) {
          if (nbr_gemm_tiny_fits(x) || !zrun_eligible(x, tk.data(), x.ntiles)) return fail(at + ": z-run item");
          const int z = x.grid[2];
          const bool six = !c.f64 && (z + 5) / 6 * 6 < (z + 7) / 8 * 8;
          if ((st.shape == 5) != six) return fail(at + ": z-run length not the one that pads z least");
          const int rz = zrun_len(st.shape, c.f64);
          const int ntx = (x.grid[0] + kBx - 1) / kBx, nty = (x.grid[1] + kBy - 1) / kBy;
          const int ntz = (z + rz - 1) / rz;
          if (g[i].gx != (unsigned)(ntx * nty * ntz) || g[i].gy != (unsigned)x.ntiles || g[i].gz != 1)
            return fail(at + ": z-run grid");
          // rows of each block as the kernel decomposes its block index
          std::vector<unsigned char> hit(rows, 0);
          for (unsigned bt = 0; bt < g[i].gx; ++bt) {
            const int ox = (bt % ntx) * kBx, oy = ((bt / ntx) % nty) * kBy, oz = (bt / (ntx * nty)) * rz;
            for (int dz = 0; dz < rz; ++dz)
              for (int dy = 0; dy < kBy; ++dy)
                for (int dx = 0; dx < kBx; ++dx) {
                  const int xx = ox + dx, yy = oy + dy, zz = oz + dz;
                  if (xx < x.grid[0] && yy < x.grid[1] && zz < z) ++hit[((long long)zz * x.grid[1] + yy) * x.grid[0] + xx];
                }
          }
          for (long long r = 0; r < rows; ++r)
            if (hit[r] != 1) return fail(at + ": z-run tiles cover a row " + std::to_string(hit[r]) + " times");
        } else {
          if (zrun_eligible(x, tk.data(), x.ntiles) || nbr_gemm_tiny_fits(x)) return fail(at + ": fallback tile form");
        }
      }
    } else if (st.kind == MK_L2L) {
      const L2lArgs* a = items<L2lArgs>(tab, st);
      int level = -1;
      for (int i = 0; i < st.n; ++i) {
        const int f = field_of(a[i].Lc);
        if (f < 0) return fail(at + ": L2L item of no field");
        const fmm_plan_t P = c.plans[f];
        int l = -1;
        for (int q = 2; q <= P->L; ++q)
          if (a[i].Lc == P->Lx(q)) l = q;
        if (l < 0) return fail(at + ": L2L writes no level");
        if (level < 0) level = l;
        if (l != level) return fail(at + ": L2L launch over two levels");
        // the field's previous L2L: level l - 1, or none before level 3 when
        // level 2 needs no harmonic rebuild
        if (!(l2l_next[f] == l - 1 || (l2l_next[f] == 1 && l == 3 && !harmonic_m2l_level(P, 2))))
          return fail(at + ": L2L out of level order");
        if (a[i].Lp != (l == 2 ? nullptr : P->Lx(l - 1))) return fail(at + ": L2L parent locals");
        if (l == P->L && fused_down(P)) return fail(at + ": leaf-level L2L outside the leaf kernel");
        l2l_next[f] = l;
      }
      if (level <= l2l_level_prev) return fail(at + ": L2L levels not coarse to fine");
      l2l_level_prev = level;
    } else if (st.kind == MK_LEAF) {
      const LeafArgs* a = items<LeafArgs>(tab, st);
      for (int i = 0; i < st.n; ++i) {
        const int f = field_of(a[i].Lleaf);
        if (f < 0) return fail(at + ": leaf item of no field");
        const fmm_plan_t P = c.plans[f];
        if (a[i].Lleaf != P->Lx(P->L) || a[i].phi != c.phi[f]) return fail(at + ": leaf buffers");
        const bool down = fused_down(P);
        if (down != (a[i].Lp != nullptr) || (down && a[i].Lp != P->Lx(P->L - 1)))
          return fail(at + ": leaf-level L2L in the leaf kernel");
        // the field's L2L chain must have reached the leaf level (the level
        // above it where the leaf kernel runs the last L2L); level 2 needs
        // none unless its locals are rebuilt from the compact rows
        const int done = l2l_next[f] == 1 && !harmonic_m2l_level(P, 2) ? 2 : l2l_next[f];
        if (done != (down ? P->L - 1 : P->L)) return fail(at + ": leaf before the field's last L2L");
        ++leaf[f];
      }
    } else if (st.kind == MK_FD) {
      for (int i = 0; i < st.n; ++i) {
        const FdArgs& x = items<FdArgs>(tab, st)[i];
        int f = -1;
        for (int q = 0; q < nf; ++q)
          if (x.phi == c.phi[q]) f = q;
        if (f < 0 || x.accel != c.acc[f] || x.nx != c.plans[f]->dims[0] || x.ny != c.plans[f]->dims[1] ||
            x.nz != c.plans[f]->dims[2])
          return fail(at + ": force item");
        ++fd[f];
      }
    }
  }
  for (int f = 0; f < nf; ++f) {
    const fmm_plan_t P = c.plans[f];
    const std::string who = "field " + std::to_string(f);
    if (p2m[f] != 1 || leaf[f] != 1 || fd[f] != (c.accel ? 1 : 0)) return fail(who + ": P2M, leaf or force count");
    if (m2m_next[f] != 2) return fail(who + ": M2M chain incomplete");
    for (int w = 2; w <= P->L + 1; ++w)
      if (gemm[f][w] != 1) return fail(who + ": contraction " + std::to_string(w) + " run " + std::to_string(gemm[f][w]) + " times");
  }
  return true;
}

// Builds the plans of one batch and its fused tables; 0 when every check
// passes.  With plant, a corruption of the built tables must be caught
// instead, each of the listed ones.
int run(bool f64, int order, int leaf, const std::vector<std::array<int, 3>>& dims, bool plant) {
  Case c;
  c.f64 = f64;
  c.accel = !f64;  // the fused form takes the stencil force in FP32 only
  for (size_t i = 0; i < dims.size(); ++i) {
    fmm_plan_t P = dry_plan(dims[i].data(), order, leaf, f64, (int)i);
    if (!P) return 1;
    c.plans.push_back(P);
    c.rho.push_back(reinterpret_cast<const void*>((uintptr_t)(i + 1) << 32));
    c.phi.push_back(reinterpret_cast<void*>(((uintptr_t)(i + 1) << 32) + ((uintptr_t)1 << 31)));
    c.acc.push_back(c.accel ? reinterpret_cast<void*>(((uintptr_t)(i + 1) << 32) + ((uintptr_t)3 << 29)) : nullptr);
  }
  fmm_batch_s B;
  B.plans = c.plans;
  if (!batch_fusable_plans(&B, c.accel)) {
    std::printf("batch: plans not fusable\n");
    return 1;
  }
  if (f64)
    build_fused<double>(&B, c.rho.data(), c.phi.data(), c.acc.data(), c.accel);
  else
    build_fused<float>(&B, c.rho.data(), c.phi.data(), c.acc.data(), c.accel);
  long long blocks = 0;
  int shapes[6] = {0, 0, 0, 0, 0, 0};
  for (const MultiStep& st : B.steps) {
    blocks += st.blocks;
    if (st.kind == MK_GEMM) shapes[st.shape] += st.n;
  }
  std::string why;
  if (!plant) {
    bool ok = check(c, B.steps, B.h_tab, &why);
    // the launch count the library reports for the batch is the schedule's
    const int reported = fmm_batch_launches(&B, c.accel ? 1 : 0);
    if (ok && reported != (int)B.steps.size()) {
      ok = false;
      why = "fmm_batch_launches reports " + std::to_string(reported);
    }
    std::printf("batch %s: %zu fields, %zu launches, %lld blocks, contraction items z-run8 %d z-run6 %d tiny %d other %d: %s\n",
                f64 ? "fp64" : "fp32", dims.size(), B.steps.size(), blocks, shapes[1], shapes[5], shapes[4],
                shapes[0] + shapes[2] + shapes[3], ok ? "ok" : why.c_str());
    return ok ? 0 : 1;
  }
  // planted corruptions, each on a fresh copy of the tables
  auto find = [&](int kind, int shape) {
    for (size_t k = 0; k < B.steps.size(); ++k)
      if (B.steps[k].kind == kind && (shape < 0 || B.steps[k].shape == shape)) return (int)k;
    return -1;
  };
  int missed = 0, tried = 0;
  auto expect_caught = [&](const char* what, std::vector<MultiStep> steps, std::vector<unsigned char> tab) {
    std::string w;
    const bool caught = !check(c, steps, tab, &w);
    std::printf("batch plant: %-52s %s%s\n", what, caught ? "caught: " : "MISSED", caught ? w.c_str() : "");
    missed += !caught;
    ++tried;
  };
  {  // a gap between two items' block ranges
    auto steps = B.steps;
    auto tab = B.h_tab;
    const int k = find(MK_P2M, -1);
    reinterpret_cast<MultiGrid*>(tab.data() + steps[k].grids_off)[1].start += 1;
    expect_caught("gap between two items' blocks", steps, tab);
  }
  {  // the launch size one block short
    auto steps = B.steps;
    const int k = find(MK_LEAF, -1);
    steps[k].blocks -= 1;
    expect_caught("launch one block short", steps, B.h_tab);
  }
  {  // a field's near field dropped from the contraction launches
    auto steps = B.steps;
    auto tab = B.h_tab;
    const int k = find(MK_GEMM, 1);
    MultiStep& st = steps[k];
    const MultiGrid* g = grids(tab, st);
    st.blocks -= (long long)g[st.n - 1].gx * g[st.n - 1].gy * g[st.n - 1].gz;
    st.n -= 1;
    expect_caught("one contraction item dropped", steps, tab);
  }
  if (find(MK_GEMM, 5) >= 0) {  // the 6-row items run with 8-row tiles
    auto steps = B.steps;
    auto tab = B.h_tab;
    MultiStep& st = steps[find(MK_GEMM, 5)];
    st.shape = 1;
    NbrGemm* a = reinterpret_cast<NbrGemm*>(tab.data() + st.args_off);
    for (int i = 0; i < st.n; ++i) a[i].shape = 1;
    expect_caught("6-row z-run items given 8-row tiles", steps, tab);
  }
  {  // a z-run item's last slab of tiles dropped
    auto steps = B.steps;
    auto tab = B.h_tab;
    MultiStep& st = steps[find(MK_GEMM, 1)];
    MultiGrid* g = reinterpret_cast<MultiGrid*>(tab.data() + st.grids_off);
    const NbrGemm* a = items<NbrGemm>(tab, st);
    for (int i = 0; i < st.n; ++i) {
      const unsigned slab = (unsigned)(((a[i].grid[0] + kBx - 1) / kBx) * ((a[i].grid[1] + kBy - 1) / kBy));
      if (g[i].gx <= slab) continue;
      const long long d = (long long)slab * g[i].gy * g[i].gz;
      g[i].gx -= slab;
      for (int j = i + 1; j < st.n; ++j) g[j].start -= d;
      st.blocks -= d;
      break;
    }
    expect_caught("z-run item without its last z slab", steps, tab);
  }
  {  // two L2L launches swapped
    auto steps = B.steps;
    const int k = find(MK_L2L, -1);
    if (k >= 0 && k + 1 < (int)steps.size() && steps[k + 1].kind == MK_L2L) {
      std::swap(steps[k], steps[k + 1]);
      expect_caught("two L2L launches swapped", steps, B.h_tab);
    }
  }
  {  // the leaf-level L2L left out of a fused leaf item
    auto steps = B.steps;
    auto tab = B.h_tab;
    const int k = find(MK_LEAF, -1);
    LeafArgs* a = reinterpret_cast<LeafArgs*>(tab.data() + steps[k].args_off);
    for (int i = 0; i < steps[k].n; ++i)
      if (a[i].Lp) {
        a[i].Lp = nullptr;
        break;
      }
    expect_caught("leaf item without its leaf-level L2L", steps, tab);
  }
  {  // the force step before the leaf evaluation
    auto steps = B.steps;
    const int k = find(MK_FD, -1), j = find(MK_LEAF, -1);
    if (k >= 0) {
      std::swap(steps[k], steps[j]);
      expect_caught("force launch before the leaf evaluation", steps, B.h_tab);
    }
  }
  {  // a contraction item reading another field's multipoles
    auto steps = B.steps;
    auto tab = B.h_tab;
    const int k = find(MK_GEMM, 1);
    NbrGemm* a = reinterpret_cast<NbrGemm*>(tab.data() + steps[k].args_off);
    std::swap(a[0].A, a[1].A);
    expect_caught("contraction items' inputs swapped", steps, tab);
  }
  std::printf("batch plant: %d of %d corruptions caught\n", tried - missed, tried);
  return missed ? 1 : 0;
}

}  // namespace batchcheck

int main(int argc, char** argv) {
  const std::string mode = argc > 1 ? argv[1] : "";
  if (mode == "batch" || mode == "batch-plant") {
    // batch fp32|fp64 ORDER LEAF NX NY NZ [NX NY NZ ...]
    if (argc < 8 || (argc - 5) % 3) return 2;
    std::vector<std::array<int, 3>> dims;
    for (int i = 5; i + 2 < argc; i += 3) dims.push_back({std::atoi(argv[i]), std::atoi(argv[i + 1]), std::atoi(argv[i + 2])});
    return batchcheck::run(std::string(argv[2]) == "fp64", std::atoi(argv[3]), std::atoi(argv[4]), dims,
                           mode == "batch-plant");
  }
  if (mode == "near4") return near4_check();
  if (mode == "centre") return centre_check();
  if (mode == "near4-protocol") return near4_protocol_check();
  if (mode == "plant") return planted_mistakes() ? 1 : 0;
  if (mode == "harmonic") return harmonic_check() ? 1 : 0;
  if (mode == "cuda-core") return cc_tiles_check() ? 1 : 0;
  if (mode == "prefix") {
    int built = 0;
    const int r = prefix_check(built);
    std::printf("prefix schedules built: %d\n", built);
    return r;
  }
  if (mode == "prefix-plant") return planted_prefix_mistakes() ? 1 : 0;
  if (mode == "rounding") return rounding_report();
  if (mode == "tables") {
    if (argc < 3) return 2;
    const std::string dir = argv[2];
    const bool ok = dump_m2l(dir, 3, 3, 3) && dump_m2l(dir, 4, 4, 4) && dump_m2l(dir, 4, 3, 4) &&
                    dump_m2l(dir, 4, 4, 3) && dump_m2p(dir, 3, 2) && dump_m2p(dir, 4, 4) && dump_m2p_grad(dir, 3, 2) && dump_m2p_grad(dir, 4, 4) && dump_near(dir, 2) &&
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
