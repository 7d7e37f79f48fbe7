// Host-side check of the LU route's step schedule (tri_analyse): for random
// triangular factors it walks the steps the way the kernel does (items of a
// step in any order, a group of 2^lg lanes per item with a butterfly sum) on
// the CPU and compares the result with plain substitution.  It also checks
// that every 16-byte staging window stays inside the padded arrays, that a
// step reads only rows finished in earlier steps and writes each row once,
// that malformed factors are rejected, that the shared-memory layout of
// lu_layout stays within its budget, and the cluster kernel's form of each
// system (lc_build).  Prints "ALL OK" on success.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "pa_internal.h"
#include "pa_lu_cluster.h"

using namespace pa;

static int g_fail = 0;
#define CHECK(c, ...)              \
  do {                             \
    if (!(c)) {                    \
      std::printf(__VA_ARGS__);    \
      std::printf("\n");           \
      g_fail = 1;                  \
      return;                      \
    }                              \
  } while (0)

struct Csr {
  int n = 0;
  std::vector<int> rp, ci;
  std::vector<double> va;
};

static Csr random_triangle(std::mt19937& g, int n, double dens, bool lower) {
  Csr T;
  T.n = n;
  T.rp.push_back(0);
  std::uniform_real_distribution<double> u(0.0, 1.0), off(-0.4, 0.4);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      const bool side = lower ? j < i : j > i;
      if (j == i) {
        T.ci.push_back(j);
        T.va.push_back((u(g) < 0.5 ? -1.0 : 1.0) * (1.5 + 3.0 * u(g)));
      } else if (side && u(g) < dens) {
        T.ci.push_back(j);
        T.va.push_back(off(g));
      }
    }
    T.rp.push_back((int)T.ci.size());
  }
  return T;
}

static void check_one(const Csr& T, bool lower) {
  const int n = T.n;
  TriHost h;
  const std::string why = tri_analyse(n, T.rp.data(), T.ci.data(), T.va.data(), lower, &h);
  CHECK(why.empty(), "analyse refused a valid factor: %s", why.c_str());
  // plain substitution
  std::mt19937 g(3);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::vector<double> b(n), ref(n), x(n);
  for (double& v : b) v = u(g);
  for (int s = 0; s < n; ++s) {
    const int i = lower ? s : n - 1 - s;
    double acc = b[i], d = 0.0;
    for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) {
      if (T.ci[k] == i) d = T.va[k];
      else acc -= T.va[k] * ref[T.ci[k]];
    }
    ref[i] = acc / d;
  }
  // the schedule, as the kernel applies it
  for (int i = 0; i < n; ++i) x[i] = b[i] * h.dinv[i];
  std::vector<int> done(n, -1);  // step in which row i received its last segment
  std::vector<int> touched(n, -1);
  const int E = (int)h.ci.size();
  for (int l = 0; l < h.nproc; ++l) {
    const int4 I = h.linfo[l];
    const int i0 = I.x, i1 = I.y & kItemMask, lg = I.y >> 27;
    CHECK(lg >= 0 && lg <= 5 && i0 <= i1 && i1 <= (int)h.items.size(), "bad step record %d", l);
    CHECK(I.z <= I.w && I.w <= E, "bad entry range at step %d", l);
    const int va0 = I.z & ~1, vb = (I.w + 1) & ~1, ca0 = I.z & ~3, cb = (I.w + 3) & ~3;
    CHECK(vb <= (int)h.va.size() && cb <= (int)h.ci.size(), "window past the padded arrays at %d", l);
    CHECK(i1 - i0 <= h.max_items && vb - va0 <= h.max_ent && cb - ca0 <= h.max_ent,
          "step %d exceeds the recorded maxima", l);
    const int G = 1 << lg;
    for (int k = i0; k < i1; ++k) {
      const int4 r = h.items[k];
      std::vector<double> lane(G, 0.0);
      int row;
      if (r.x >= 0) {  // one entry: {row, column, value}
        row = r.x;
        CHECK(r.y >= 0 && r.y < n && done[r.y] < l, "step %d reads unfinished x[%d]", l, r.y);
        double v;
        const int w[2] = {r.z, r.w};
        std::memcpy(&v, w, sizeof v);
        lane[0] = std::fma(v, x[r.y], x[row]);
      } else {  // {~row, first entry, end entry}
        row = ~r.x;
        CHECK(r.y >= I.z && r.z <= I.w && r.z - r.y >= 2, "bad segment at step %d", l);
        lane[0] = x[row];
        for (int gl = 0; gl < G; ++gl)
          for (int e = r.y + gl; e < r.z; e += G) {
            const int c = h.ci[e];
            CHECK(c >= 0 && c < n && done[c] < l, "step %d reads unfinished x[%d]", l, c);
            lane[gl] = std::fma(h.va[e], x[c], lane[gl]);
          }
      }
      CHECK(row >= 0 && row < n, "row out of range at step %d", l);
      CHECK(touched[row] != l, "row %d written twice in step %d", row, l);
      touched[row] = l;
      for (int d = G >> 1; d > 0; d >>= 1) {
        std::vector<double> nx(G);
        for (int q = 0; q < G; ++q) nx[q] = lane[q] + lane[q ^ d];
        lane = nx;
      }
      x[row] = lane[0];
    }
    for (int i = 0; i < n; ++i)
      if (touched[i] == l) done[i] = l;
  }
  double err = 0.0, nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    err = std::fmax(err, std::fabs(x[i] - ref[i]));
    nrm = std::fmax(nrm, std::fabs(ref[i]));
  }
  CHECK(err <= 1e-12 * (nrm > 0 ? nrm : 1.0), "n=%d lower=%d: |x - ref| = %.3e of %.3e", n, lower,
        err, nrm);
}

// lc_build: the cluster form of a system for 2^lgC CTAs in batches of at
// most cap records.  Every step's items are split by owning CTA (row mod C)
// without loss or duplication, the batches tile each CTA's steps and stream
// run, and replaying the steps CTA by CTA, lanes and butterflies included,
// gives plain substitution.
static void check_cluster(const Csr& T, bool lower, int lgC, int cap) {
  const int n = T.n, C = 1 << lgC;
  TriHost h;
  CHECK(tri_analyse(n, T.rp.data(), T.ci.data(), T.va.data(), lower, &h).empty(), "analyse failed");
  LcHost c;
  lc_build(h, lgC, cap, &c);
  CHECK(c.nproc == h.nproc && c.bbase.size() == (size_t)C + 1 && c.bbase[0] == 0 &&
            c.bbase[C] == (int)c.batch.size(), "cluster form: batch index");
  std::mt19937 g(5);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::vector<double> b(n), ref(n), x(n);
  for (double& v : b) v = u(g);
  for (int s = 0; s < n; ++s) {
    const int i = lower ? s : n - 1 - s;
    double acc = b[i], d = 0.0;
    for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) {
      if (T.ci[k] == i) d = T.va[k];
      else acc -= T.va[k] * ref[T.ci[k]];
    }
    ref[i] = acc / d;
  }
  for (int i = 0; i < n; ++i) x[i] = b[i] * h.dinv[i];
  CHECK(c.fin0.size() == (size_t)n, "cluster form: fin0 size");
  // batches: consecutive steps, contiguous stream runs, within cap unless alone
  size_t total = 0;
  for (int cb = 0; cb < C; ++cb) {
    int step = 0, off = -1;
    for (int k = c.bbase[cb]; k < c.bbase[cb + 1]; ++k) {
      const int4 bt = c.batch[k];
      CHECK(bt.x == step && bt.y > bt.x && (off < 0 || bt.z == off), "CTA %d batch %d does not follow", cb, k);
      CHECK(bt.w <= cap || bt.y == bt.x + 1, "CTA %d batch %d: %d records over the cap %d", cb, k, bt.w, cap);
      CHECK(bt.z >= 0 && (size_t)bt.z + bt.w <= c.stream.size(), "CTA %d batch %d outside the stream", cb, k);
      step = bt.y;
      off = bt.z + bt.w;
      total += bt.w;
    }
    CHECK(step == c.nproc, "CTA %d: batches end at step %d of %d", cb, step, c.nproc);
  }
  CHECK(total == c.stream.size(), "cluster form: stream holds %zu records, batches %zu", c.stream.size(), total);
  // the replay, step by step across CTAs
  std::vector<int> bi(C), pos(C, 0);
  for (int cb = 0; cb < C; ++cb) bi[cb] = c.bbase[cb];
  std::vector<int> done(n, -1), touched(n, -1), marked(n, -1), seen(n, -1);
  for (int l = 0; l < c.nproc; ++l) {
    int step_items = 0;
    for (int cb = 0; cb < C; ++cb) {
      if (l == c.batch[bi[cb]].y) {
        ++bi[cb];
        pos[cb] = 0;
      }
      const int4 bt = c.batch[bi[cb]];
      CHECK(bt.x <= l && l < bt.y, "step %d CTA %d: not in its batch", l, cb);
      const int4* blk = c.stream.data() + bt.z + pos[cb];
      const int4 hd = blk[0];
      const int cnt = hd.x & kItemMask, lg = hd.x >> 27, G = 1 << lg, ne = hd.y;
      CHECK(lg >= 0 && lg <= 5 && cnt >= 0 && ne >= 0 && hd.z == 0 && hd.w == 0, "step %d CTA %d: bad header", l, cb);
      CHECK(pos[cb] + 1 + cnt + ne <= bt.w, "step %d CTA %d: block past its batch", l, cb);
      step_items += cnt;
      int seg_ent = 0;
      for (int k = 1; k <= cnt; ++k) {
        const int4 r = blk[k];
        std::vector<double> lane(G, 0.0);
        int row;
        bool last;
        if (r.x >= 0) {
          row = r.x & kItemMask;
          last = (r.x & kLcLast) != 0;
          CHECK((r.x & ~(kItemMask | kLcLast)) == 0, "step %d CTA %d: bad row word", l, cb);
          CHECK(r.y >= 0 && r.y < n && done[r.y] < l, "step %d reads unfinished x[%d]", l, r.y);
          double v;
          const int w[2] = {r.z, r.w};
          std::memcpy(&v, w, sizeof v);
          lane[0] = std::fma(v, x[r.y], x[row]);
        } else {
          row = ~r.x;
          last = r.w != 0;
          CHECK(r.w == 0 || r.w == 1, "step %d CTA %d: bad segment mark", l, cb);
          CHECK(r.y >= 1 + cnt && r.z <= 1 + cnt + ne && r.z - r.y >= 2, "step %d CTA %d: segment outside the block", l, cb);
          seg_ent += r.z - r.y;
          lane[0] = x[row];
          for (int gl = 0; gl < G; ++gl)
            for (int e = r.y + gl; e < r.z; e += G) {
              const int4 q = blk[e];
              double v;
              const int w[2] = {q.z, q.w};
              std::memcpy(&v, w, sizeof v);
              CHECK(q.x >= 0 && q.x < n && done[q.x] < l, "step %d reads unfinished x[%d]", l, q.x);
              lane[gl] = std::fma(v, x[q.x], lane[gl]);
            }
        }
        CHECK(row >= 0 && row < n && (row & (C - 1)) == cb, "step %d: row %d applied by CTA %d", l, row, cb);
        CHECK(touched[row] != l, "row %d written twice in step %d", row, l);
        CHECK(marked[row] < 0, "row %d has an item after its last", row);
        touched[row] = l;
        seen[row] = l;
        if (last) marked[row] = l;
        for (int d = G >> 1; d > 0; d >>= 1) {
          std::vector<double> nx(G);
          for (int q = 0; q < G; ++q) nx[q] = lane[q] + lane[q ^ d];
          lane = nx;
        }
        x[row] = lane[0];
      }
      CHECK(seg_ent == ne, "step %d CTA %d: %d entries used of %d", l, cb, seg_ent, ne);
      pos[cb] += 1 + cnt + ne;
    }
    const int4 I = h.linfo[l];
    CHECK(step_items == (I.y & kItemMask) - I.x, "step %d: %d items, step form %d", l, step_items,
          (I.y & kItemMask) - I.x);
    for (int i = 0; i < n; ++i)
      if (touched[i] == l) done[i] = l;
  }
  for (int i = 0; i < n; ++i) {  // a last mark on every row with items, fin0 on the others
    CHECK(marked[i] == seen[i], "row %d: last item in step %d, marked in %d", i, seen[i], marked[i]);
    CHECK((c.fin0[i] != 0) == (seen[i] < 0), "row %d: fin0 %d, items %d", i, c.fin0[i], seen[i] >= 0);
  }
  double err = 0.0, nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    err = std::fmax(err, std::fabs(x[i] - ref[i]));
    nrm = std::fmax(nrm, std::fabs(ref[i]));
  }
  CHECK(err <= 1e-12 * (nrm > 0 ? nrm : 1.0), "cluster n=%d lower=%d C=%d cap=%d: |x - ref| = %.3e of %.3e",
        n, lower, C, cap, err, nrm);
}

static void check_rejections() {
  const int rp[3] = {0, 1, 3};
  const int ci_zero[3] = {0, 0, 1};
  const double va_zero[3] = {2.0, 1.0, 0.0};  // zero diagonal in row 1
  TriHost h;
  CHECK(!tri_analyse(2, rp, ci_zero, va_zero, true, &h).empty(), "zero diagonal accepted");
  const int ci_up[3] = {0, 1, 1};  // row 1 holds (1, 1) twice
  const double va_up[3] = {2.0, 1.0, 3.0};
  CHECK(!tri_analyse(2, rp, ci_up, va_up, true, &h).empty(), "two diagonals accepted");
  const int rp2[3] = {0, 2, 3};
  const int ci_side[3] = {0, 1, 1};  // (0, 1) above the diagonal of a lower factor
  const double va_side[3] = {2.0, 1.0, 3.0};
  CHECK(!tri_analyse(2, rp2, ci_side, va_side, true, &h).empty(), "entry above the diagonal accepted");
  CHECK(tri_analyse(2, rp2, ci_side, va_side, false, &h).empty(), "valid upper factor refused");
}

// lu_layout: the dynamic shared memory it asks for stays within the budget,
// the slots keep 16-byte alignment, and the solve vector goes to shared
// memory exactly when it fits beside a minimal ring.
static void check_layout() {
  const int ns[] = {1, 7, 294, 2646, 10086, 26000, 40000};
  const int wins[] = {1, 64, 500, 3000, 20000};
  for (int n : ns)
    for (int wi : wins) {
      LuParams p{};
      p.n = n;
      TriSys t{};
      t.max_items = wi;
      t.max_ent = wi + 3;
      p.L = p.U = p.Ut = p.Lt = t;
      const size_t smem = lu_layout(&p);
      CHECK(smem <= kLuSmemBudget, "n=%d win=%d: %zu bytes over the budget", n, wi, smem);
      CHECK(p.slot_items > 0 && p.slot_ent > 0 && p.slot_ent % 4 == 0, "n=%d win=%d: bad slot caps", n, wi);
      const size_t slot = 32 + 16 * (size_t)p.slot_items + 12 * (size_t)p.slot_ent;
      CHECK(slot % 16 == 0, "n=%d: slot of %zu bytes breaks 16-byte alignment", n, slot);
      const size_t vec = sizeof(double) * ((size_t)n + (n & 1));
      CHECK((p.smem_mode == 1) == (smem > vec && vec + 7 * (32 + 20 * 64) <= kLuSmemBudget),
            "n=%d win=%d: solve-vector placement", n, wi);
      CHECK(smem == (p.smem_mode == 1 ? vec : 0) + 7 * slot, "n=%d win=%d: size mismatch", n, wi);
      if (p.slot_items >= wi && p.slot_ent >= ((wi + 3 + 3) & ~3)) continue;
      // capped: the ring then uses (nearly) all of what is left
      const size_t left = kLuSmemBudget - (p.smem_mode == 1 ? vec : 0);
      CHECK(7 * slot + 7 * (16 + 12 * 4 + 16) >= left / 2, "n=%d win=%d: ring needlessly small", n, wi);
    }
}

int main() {
  std::mt19937 g(11);
  const int sizes[] = {1, 2, 5, 33, 64, 150, 300};
  const double dens[] = {0.0, 0.02, 0.1, 0.4, 1.0};
  for (int n : sizes)
    for (double d : dens)
      for (int lower = 0; lower < 2; ++lower) {
        const Csr T = random_triangle(g, n, d, lower != 0);
        check_one(T, lower != 0);
        for (int lgC = 3; lgC <= 4; ++lgC)
          for (int cap : {4, 40, 1280}) check_cluster(T, lower != 0, lgC, cap);
        if (g_fail) return 1;
      }
  check_rejections();
  if (g_fail) return 1;
  check_layout();
  if (g_fail) return 1;
  std::printf("ALL OK\n");
  return 0;
}
