// The level passes of paper_1110_2477_gb300/csrc (ob_tc.cuh, ob_adj.cuh, ob_path.cuh) compiled
// for the host with a one-lane team, for CPU tests of their logic: pricing (TcRun), the split
// of a level over G teams (TcGroup, run phase by phase), the adjoint (TcAdj), the hedge at
// the root (TcRun::root_hedge) and the hedge along a path (path_one).  Test
// infrastructure only; the library itself runs these passes on the GPU.
#include <cstring>
#include <vector>

#include "ob_adj.cuh"
#include "ob_path.cuh"

namespace {

struct OneLane {
  static constexpr int W = 1;
  int lane() const { return 0; }
  void sync() const {}
  template <class T> T bcast0(T v) const { return v; }
  template <class T> T prev(T, T carry) const { return carry; }
  template <class T> T prev_last(T v, T carry, T& last) const { last = v; return carry; }
  int count_le(int v, int q) const { return v <= q; }
  void count_le2(int v, int q1, int q2, int& c1, int& c2) const { c1 = v <= q1; c2 = v <= q2; }
  template <class T> void look2(T v, T c1, T c2, T& m1, T& m2, T& l1, T& l2) const {
    m1 = c1; m2 = c2; l1 = v; l2 = c1;
  }
  int count(bool p) const { return p; }
  bool any(bool p) const { return p; }
  int excl_sum(int v, int& total) const { total = v; return 0; }
  long long seg_min(long long v, bool head, long long& carry) const {
    const long long r = head ? v : (v < carry ? v : carry);
    carry = r;
    return r;
  }
  void seg_argmin(long long& v, int& ix, bool head, long long& cv, int& ci) const {
    if (!head && cv < v) { v = cv; ix = ci; }
    cv = v;
    ci = ix;
  }
  template <class T> T sum(T v) const { return v; }
};

std::vector<char> g_arena;

char* arena(size_t bytes) {
  if (g_arena.size() < bytes) g_arena.resize(bytes);
  return g_arena.data();
}

}  // namespace

// The pricing run plus the hedge at the root (TcRun::root_hedge): hedge[4] as the library
// returns it (holdings of the seller and the buyer, the two exercise flags).
extern "C" int hp_price_hedge(const obk::Opt* o, double* out, double* hedge) {
  const size_t bytes = 256ull << 20;
  OneLane tm;
  obk::Lay L;
  if (!obk::carve(arena(bytes), bytes, o->N, 16, L)) return obk::ST_CAPACITY;
  obk::TcRun<OneLane> R(tm, *o, L);
  const int rc = R.run(out[0], out[1]);
  for (int c = 0; c < 4; ++c) hedge[c] = R.st.hedge[c];
  return rc;
}

extern "C" int hp_price(const obk::Opt* o, double* out, long long* pts) {
  const size_t bytes = 256ull << 20;
  OneLane tm;
  obk::Lay L;
  if (!obk::carve(arena(bytes), bytes, o->N, 16, L)) return obk::ST_CAPACITY;
  obk::TcRun<OneLane> R(tm, *o, L);
  const int rc = R.run(out[0], out[1]);
  pts[0] = R.st.upts;
  pts[1] = R.st.wpts;
  pts[2] = R.st.zpts;
  return rc;
}

// The fused level step (TcRun::level_fused): w of chunks of whole nodes in an array of
// `cap` points (shared memory on the GPU; here host memory poisoned with NaN).
extern "C" int hp_price_chip(const obk::Opt* o, int cap, double* out, long long* pts) {
  const size_t bytes = 256ull << 20;
  OneLane tm;
  obk::Lay L;
  if (!obk::carve(arena(bytes), bytes, o->N, 16, L)) return obk::ST_CAPACITY;
  std::vector<char> chip((size_t)cap * obk::WBUF_POINT_BYTES + 64);
  std::memset(chip.data(), 0xff, chip.size());
  obk::TcRun<OneLane, true> R(tm, *o, L);
  R.chip = obk::carve_wbuf(chip.data(), cap);
  const int rc = R.run(out[0], out[1]);
  pts[0] = R.st.upts;
  pts[1] = R.st.wpts;
  pts[2] = R.st.zpts;
  return rc;
}

extern "C" int hp_price_split(const obk::Opt* o, int G, double* out, long long* pts) {
  const size_t shared_bytes = 64ull << 20, priv_bytes = 32ull << 20;
  char* base = arena(shared_bytes + priv_bytes * (size_t)G);
  std::memset(base, 0xff, shared_bytes + priv_bytes * (size_t)G);  // NaN: stale data shows
  OneLane tm;
  obk::GroupLay S;
  if (!obk::carve_group_shared(base, shared_bytes, o->N, 2 * (o->N + 2), S)) return obk::ST_CAPACITY;
  std::vector<obk::Lay> Lp(G);
  std::vector<obk::TcGroup<OneLane>*> team(G);
  for (int c = 0; c < G; ++c) {
    if (!obk::carve(base + shared_bytes + priv_bytes * (size_t)c, priv_bytes, o->N, 16, Lp[c]))
      return obk::ST_CAPACITY;
    team[c] = new obk::TcGroup<OneLane>(tm, *o, Lp[c], S, G, c);
  }
  int rc = team[0]->begin();
  for (int c = 1; c < G; ++c) team[c]->begin();
  std::vector<int> cnt(G);
  for (int t = o->N; t >= 0 && rc == obk::ST_OK; --t) {
    for (int c = 0; c < G; ++c) cnt[c] = team[c]->compute(t) ? team[c]->ztot : -1;
    for (int c = 0; c < G; ++c)
      if (cnt[c] < 0) rc = obk::ST_CAPACITY;
    for (int c = 0; c < G && rc == obk::ST_OK; ++c)
      if (!team[c]->publish(t, cnt.data())) rc = obk::ST_CAPACITY;
  }
  if (rc == obk::ST_OK) team[0]->root(out[0], out[1]);
  pts[0] = pts[1] = pts[2] = 0;
  for (int c = 0; c < G; ++c) {
    pts[0] += team[c]->R.st.upts;
    pts[1] += team[c]->R.st.wpts;
    pts[2] += team[c]->R.st.zpts;
    delete team[c];
  }
  return rc;
}

// The whole-GPU form's level loop with trapezoid rounds (TcTrap) for light levels, G teams
// run phase by phase over NaN-poisoned scratch: a level B whose points are at most
// light_points * G goes down up to Dmax levels in one round, otherwise one level (TcGroup).
// rounds[0] counts the trapezoid rounds, rounds[1] the single levels.
extern "C" int hp_price_trap(const obk::Opt* o, int G, int Dmax, int light_points, int column_points,
                             double* out, long long* pts, int* rounds) {
  const size_t shared_bytes = 64ull << 20, priv_bytes = 32ull << 20;
  char* base = arena(shared_bytes + priv_bytes * (size_t)G);
  std::memset(base, 0xff, shared_bytes + priv_bytes * (size_t)G);
  OneLane tm;
  obk::GroupLay S;
  if (!obk::carve_group_shared(base, shared_bytes, o->N, 2 * (o->N + 2), S)) return obk::ST_CAPACITY;
  std::vector<obk::Lay> Lp(G);
  std::vector<obk::TcGroup<OneLane>*> team(G);
  std::vector<obk::TcTrap<OneLane>*> trap(G);
  for (int c = 0; c < G; ++c) {
    if (!obk::carve(base + shared_bytes + priv_bytes * (size_t)c, priv_bytes, o->N, 16, Lp[c]))
      return obk::ST_CAPACITY;
    team[c] = new obk::TcGroup<OneLane>(tm, *o, Lp[c], S, G, c);
    trap[c] = new obk::TcTrap<OneLane>(tm, *o, Lp[c], S);
  }
  int rc = team[0]->begin();
  for (int c = 1; c < G; ++c) team[c]->begin();
  std::vector<int> cnt(G), cnt2(G);
  rounds[0] = rounds[1] = 0;
  for (int t = o->N; t >= 0 && rc == obk::ST_OK;) {
    const int B = t + 1;
    const long long zb = S.off[B & 1][2 * (B + 1)];
    if (zb <= (long long)light_points * G && zb <= (long long)column_points * (B + 1)) {
      int D = 0, Ga = 0;
      for (int c = 0; c < G; ++c) {
        int a, b;
        trap[c]->plan(B, Dmax, G, c, D, Ga, a, b);
        const bool ok = trap[c]->compute(B, D, a, b);
        cnt[c] = ok ? trap[c]->nS : -1;
        cnt2[c] = ok ? trap[c]->nB : 0;
        if (!ok) rc = obk::ST_CAPACITY;
      }
      for (int c = 0; c < G && rc == obk::ST_OK; ++c)
        if (!trap[c]->publish(B - D, G, c, cnt.data(), cnt2.data())) rc = obk::ST_CAPACITY;
      ++rounds[0];
      t = B - D - 1;
      continue;
    }
    for (int c = 0; c < G; ++c) cnt[c] = team[c]->compute(t) ? team[c]->ztot : -1;
    for (int c = 0; c < G; ++c)
      if (cnt[c] < 0) rc = obk::ST_CAPACITY;
    for (int c = 0; c < G && rc == obk::ST_OK; ++c)
      if (!team[c]->publish(t, cnt.data())) rc = obk::ST_CAPACITY;
    ++rounds[1];
    --t;
  }
  if (rc == obk::ST_OK) team[0]->root(out[0], out[1]);
  pts[0] = pts[1] = pts[2] = 0;
  for (int c = 0; c < G; ++c) {
    pts[0] += team[c]->R.st.upts + trap[c]->R.st.upts;
    delete team[c];
    delete trap[c];
  }
  return rc;
}

// Every level with its nodes split over G teams at the G-quantiles of the merged successor
// points (TcSplit), the teams run phase by phase over NaN-poisoned scratch.
extern "C" int hp_price_nsplit(const obk::Opt* o, int G, double* out, long long* pts) {
  const size_t shared_bytes = 64ull << 20, priv_bytes = 32ull << 20;
  char* base = arena(shared_bytes + priv_bytes * (size_t)G);
  std::memset(base, 0xff, shared_bytes + priv_bytes * (size_t)G);
  OneLane tm;
  obk::GroupLay S;
  if (!obk::carve_group_shared(base, shared_bytes, o->N, 2 * (o->N + 2), S)) return obk::ST_CAPACITY;
  std::vector<obk::Lay> Lp(G);
  std::vector<obk::TcSplit<OneLane>*> team(G);
  for (int c = 0; c < G; ++c) {
    if (!obk::carve(base + shared_bytes + priv_bytes * (size_t)c, priv_bytes, o->N, 16, Lp[c]))
      return obk::ST_CAPACITY;
    team[c] = new obk::TcSplit<OneLane>(tm, *o, Lp[c], S, G, c);
  }
  obk::TcGroup<OneLane> g0(tm, *o, Lp[0], S, G, 0);
  int rc = g0.begin();  // the leaves, and every team's tree constants
  for (int c = 1; c < G; ++c) obk::TcGroup<OneLane>(tm, *o, Lp[c], S, G, c).begin();
  std::vector<obk::SplitRec> recs(G);
  std::vector<int> cnt(G);
  for (int t = o->N; t >= 0 && rc == obk::ST_OK; --t) {
    for (int c = 0; c < G; ++c) team[c]->phase_a(t, recs.data());
    if (obk::TcSplit<OneLane>::overflow(recs.data(), G)) { rc = obk::ST_CAPACITY; break; }
    for (int c = 0; c < G; ++c) team[c]->phase_b(recs.data());
    for (int c = 0; c < G; ++c) cnt[c] = team[c]->phase_c(t, recs.data()) ? team[c]->ztot : -1;
    for (int c = 0; c < G; ++c)
      if (cnt[c] < 0) rc = obk::ST_CAPACITY;
    for (int c = 0; c < G && rc == obk::ST_OK; ++c)
      if (!team[c]->publish(t, cnt.data())) rc = obk::ST_CAPACITY;
  }
  if (rc == obk::ST_OK) g0.root(out[0], out[1]);
  pts[0] = pts[1] = pts[2] = 0;
  for (int c = 0; c < G; ++c) {
    pts[0] += team[c]->R.st.upts;
    pts[1] += team[c]->R.st.wpts;
    pts[2] += team[c]->R.st.zpts;
    delete team[c];
  }
  return rc;
}

// full = 1: the records of every level kept by the forward pass; 0: checkpoints and a
// recomputed segment per checkpoint
extern "C" int hp_greeks(const obk::Opt* o, double* out, double* grad, int full) {
  const size_t bytes = 512ull << 20;
  OneLane tm;
  obk::Lay L;
  obk::AdjLay A;
  if (!obk::carve_greeks(arena(bytes), bytes, o->N, 2 * (o->N + 2), L, A, full != 0))
    return obk::ST_CAPACITY;
  obk::TcRun<OneLane> R(tm, *o, L);
  obk::TcAdj<OneLane> G(R, A);
  return G.run(out[0], out[1], grad, grad + obk::NPAR, full != 0);
}

// The hedge along a path (path_one) for one checked option: out = (ask, bid), hold and cash
// 2 (N+1) doubles each, *stop the buyer's stopping level.  slice_kb: the option's scratch.
extern "C" int hp_hedge_path(const obk::Opt* o, const int8_t* moves, int slice_kb, double* out, double* hold,
                             double* cash, int* stop) {
  const size_t bytes = (size_t)slice_kb << 10;
  OneLane tm;
  return obk::path_one(tm, *o, moves, arena(bytes), bytes, out[0], out[1], hold, cash, *stop);
}
