// Compiles a LoLa layer list (paper Sec. 4.2-4.4, Tables 1 and 3) into waves
// of batched ciphertext operations and runs them.
//
// Every layer is expressed with five batched ops: scalar multiply-accumulate
// (convolution row-major), rotation waves (with an optional fused
// accumulate: x + rot(x, s) is one key switch + one add in the same
// kernel), message sums, ct x plaintext and square (ct (x) ct +
// relinearisation).  Independent rotations of one layer (the rounds of a
// stacked row-major product, the outputs of an interleaved row-major
// product, the messages being combined) run in the same wave, so one launch
// carries many ciphertexts and one key read serves all of them.
#include <string.h>

#include <algorithm>
#include <map>
#include <set>

#include "net.h"

namespace lola {

#define TRY(x)                      \
  do {                              \
    int _rc = (x);                  \
    if (_rc != LOLA_OK) return _rc; \
  } while (0)

// ------------------------------------------------------------ compile state
struct Repr {
  lola_repr kind = LOLA_REPR_DENSE;
  int reg = -1;
  uint32_t msgs = 0;
  std::vector<std::pair<uint32_t, uint32_t>> pos;   // element -> (message, slot)
  uint32_t block = 0, copies = 0;
};

struct Builder {
  Ctx* c;                                  // full context
  Net* net;
  uint32_t level = 0;                      // ciphertext primes of the current messages
  Ctx* lc = nullptr;                       // context of that level
  std::map<uint32_t, std::vector<std::vector<int64_t>>> pts;   // level -> plaintext slot vectors
  std::vector<uint64_t> w, ws;             // MAC tables
  std::set<int32_t> steps;

  int vreg(uint32_t msgs) {
    net->vreg_msgs.push_back(msgs);
    net->vreg_level.push_back(level);
    return (int)net->vreg_msgs.size() - 1;
  }
  // dst[0..k) = (accum ? accum : 0) + rot(src, step_i)
  void rot(int dst, int src, int accum, uint32_t msgs, const std::vector<int32_t>& st) {
    Op o;
    o.kind = OP_ROT;
    o.dst = dst;
    o.src = src;
    o.aux = accum;
    o.msgs = msgs;
    o.steps = st;
    for (int32_t s : st) steps.insert(s);
    net->ops.push_back(o);
  }
  // x <- x + rot(x, s) for s in shifts (0 = row swap), on all `msgs`
  // messages of x.  hoist = m > 1: runs of up to m consecutive nonzero
  // shifts a_1 .. a_r (r > 1) become one rotate-sum over the 2^r - 1 subset
  // sums (sum_{i in S} a_i mod n/2, S as a bit mask, ascending), which adds
  // the same rotations of x in one key switch; a row swap, a lone shift, or
  // a run with a subset sum of 0 mod n/2 stays x + rot(x, s) per step.
  int rotate_and_sum(int x, uint32_t msgs, const std::vector<int32_t>& shifts, uint32_t hoist = 1) {
    const uint32_t h = c->n / 2;
    std::vector<int32_t> run;
    auto single = [&](int32_t s) {
      const int y = vreg(msgs);
      rot(y, x, x, msgs, std::vector<int32_t>(msgs, s));
      x = y;
    };
    auto flush = [&]() {
      if (run.empty()) return;
      std::vector<int32_t> sums;
      bool zero = false;
      for (uint32_t mask = 1; mask < (1u << run.size()); ++mask) {
        uint64_t t = 0;
        for (size_t i = 0; i < run.size(); ++i)
          if (mask >> i & 1) t += (uint64_t)run[i];
        t %= h;
        zero |= t == 0;
        sums.push_back((int32_t)t);
      }
      if (run.size() == 1 || zero) {
        for (int32_t s : run) single(s);
      } else {
        Op o;
        o.kind = OP_ROT_SUM;
        o.src = x;
        o.dst = vreg(msgs);
        o.msgs = msgs;
        o.steps = sums;
        for (int32_t s : sums) steps.insert(s);
        net->ops.push_back(o);
        x = o.dst;
      }
      run.clear();
    };
    for (int32_t s : shifts) {
      if (s == 0) {
        flush();
        single(0);
        continue;
      }
      run.push_back(s);
      if (run.size() >= std::max<uint32_t>(hoist, 1)) flush();
    }
    flush();
    return x;
  }
  size_t add_plaintexts(const std::vector<std::vector<int64_t>>& v) {
    auto& lv = pts[level];
    const size_t first = lv.size();
    for (auto& p : v) lv.push_back(p);
    return first;
  }
};

static int layer_conv(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n;
  if (r.kind != LOLA_REPR_CONVOLUTION) return fail(LOLA_E_REPR, "conv layer needs the convolution representation");
  if (!L.weights || L.cols != r.msgs || L.rows == 0) return fail(LOLA_E_PARAM, "conv weights must be maps x window");
  const uint32_t maps = L.rows, R = L.cols;
  Op o;
  o.kind = OP_MAC;
  o.src = r.reg;
  o.dst = b.vreg(maps);
  o.msgs = maps;
  o.R = R;
  o.w_first = b.w.size();
  const uint32_t kt = b.c->kt, Lq = b.level;   // the table holds the current level's primes
  // table order [R][kt][L][maps]: the maps a thread accumulates sit together
  for (uint32_t j = 0; j < R; ++j)
    for (uint32_t ti = 0; ti < kt; ++ti) {
      const int64_t t = (int64_t)b.c->primes[b.c->iT() + ti];
      for (uint32_t l = 0; l < Lq; ++l) {
        const uint64_t q = b.c->primes[l];
        for (uint32_t m = 0; m < maps; ++m) {
          int64_t v = L.weights[(size_t)m * R + j] % t;   // centered lift mod t (Sec. 3.1 scalar)
          if (v < 0) v += t;
          if (v > (t - 1) / 2) v -= t;
          const uint64_t x = v >= 0 ? (uint64_t)v % q : (q - ((uint64_t)(-v) % q)) % q;
          b.w.push_back(x);
          b.ws.push_back(shoup_h(x, q));
        }
      }
    }
  b.net->ops.push_back(o);
  const uint32_t width = (uint32_t)r.pos.size();
  Repr out;
  out.kind = LOLA_REPR_DENSE;
  out.reg = o.dst;
  out.msgs = maps;
  for (uint32_t m = 0; m < maps; ++m)
    for (uint32_t i = 0; i < width; ++i) out.pos.push_back({m, r.pos[i].second});
  for (auto& p : out.pos)
    if (p.second >= n) return fail(LOLA_E_PARAM, "slot out of range");
  r = out;
  return LOLA_OK;
}

// Dense -> convolution representation by masking (App. C, LoLa-Dense):
// weights[r][e] = input element that message r holds at element e (-1 =
// zero padding).  Message 0 keeps its elements at their input slots S_e;
// message r must be one shift off_r of message 0.  The input is rotated
// left by every off_r in one hoisted rotation (one decomposition for all),
// then each message is multiplied by the 0/1 mask of its elements' slots.
static int layer_masked_shifts(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n, h = n / 2;
  if (r.kind != LOLA_REPR_DENSE || r.msgs != 1) return fail(LOLA_E_REPR, "masked shifts need one dense message");
  for (auto& p : r.pos)
    if (p.first != 0) return fail(LOLA_E_REPR, "masked shifts need one dense message");
  const uint32_t R = L.rows, E = L.cols;
  if (!L.weights || R == 0 || E == 0) return fail(LOLA_E_PARAM, "masked shifts need a messages x elements gather");
  auto G = [&](uint32_t m, uint32_t e) { return L.weights[(size_t)m * E + e]; };
  std::vector<uint32_t> S(E);
  for (uint32_t e = 0; e < E; ++e) {
    const int64_t g = G(0, e);
    if (g < 0 || (uint64_t)g >= r.pos.size()) return fail(LOLA_E_PARAM, "message 0 must hold every element");
    S[e] = r.pos[(size_t)g].second;
    if (S[e] >= h) return fail(LOLA_E_PARAM, "masked shifts: elements must sit in slot row 0");
  }
  std::vector<uint32_t> off(R, 0);
  std::set<uint32_t> seen;
  for (uint32_t m = 0; m < R; ++m) {
    bool have = false;
    int64_t o = 0;
    for (uint32_t e = 0; e < E; ++e) {
      const int64_t g = G(m, e);
      if (g < 0) continue;
      if ((uint64_t)g >= r.pos.size()) return fail(LOLA_E_PARAM, "gather index out of range");
      const int64_t d = (int64_t)r.pos[(size_t)g].second - (int64_t)S[e];
      if (have && d != o) return fail(LOLA_E_PARAM, "message is not one shift of message 0");
      o = d;
      have = true;
    }
    if (!have || o < 0 || o >= (int64_t)h || ((m == 0) != (o == 0)))
      return fail(LOLA_E_PARAM, "masked shifts: offsets must be 0 for message 0, else in (0, n/2)");
    off[m] = (uint32_t)o;
    if (!seen.insert(off[m]).second) return fail(LOLA_E_PARAM, "masked shifts: offsets must be distinct");
    for (uint32_t e = 0; e < E; ++e)
      if (S[e] + off[m] >= h) return fail(LOLA_E_PARAM, "masked shifts would wrap a slot row");
  }
  std::vector<std::vector<int64_t>> M(R, std::vector<int64_t>(n, 0));
  for (uint32_t m = 0; m < R; ++m)
    for (uint32_t e = 0; e < E; ++e)
      if (G(m, e) >= 0) M[m][S[e]] = 1;
  const int outr = b.vreg(R);
  const size_t pt0 = b.add_plaintexts(M);
  Op m0;                                    // message 0: x * mask_0, straight into the output
  m0.kind = OP_MULPT;
  m0.src = r.reg;
  m0.src_stride = 0;
  m0.dst = outr;
  m0.msgs = 1;
  m0.pt_first = pt0;
  b.net->ops.push_back(m0);
  if (R > 1) {
    Op ro;                                  // messages 1..R-1: x rotated left by off_r, hoisted
    ro.kind = OP_ROT_HOISTED;
    ro.src = r.reg;
    ro.dst = b.vreg(R - 1);
    ro.msgs = R - 1;
    for (uint32_t m = 1; m < R; ++m) ro.steps.push_back((int32_t)(h - off[m]));   // left by off = right by h - off
    for (int32_t s : ro.steps) b.steps.insert(s);
    b.net->ops.push_back(ro);
    Op mr;                                  // then times mask_r
    mr.kind = OP_MULPT;
    mr.src = ro.dst;
    mr.src_stride = 1;
    mr.dst = outr;
    mr.dst_off = 1;
    mr.msgs = R - 1;
    mr.pt_first = pt0 + 1;
    b.net->ops.push_back(mr);
  }
  Repr out;
  out.kind = LOLA_REPR_CONVOLUTION;
  out.reg = outr;
  out.msgs = R;
  for (uint32_t e = 0; e < E; ++e) out.pos.push_back({0, S[e]});
  r = out;
  return LOLA_OK;
}

static int layer_combine(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t h = b.c->n / 2;
  if (r.kind != LOLA_REPR_DENSE && r.kind != LOLA_REPR_INTERLEAVED)
    return fail(LOLA_E_REPR, "combine needs dense messages");
  // shifts: weights (1 x messages, shift[0] = 0) or m * stride
  std::vector<uint64_t> shift(r.msgs);
  if (L.weights) {
    if (L.rows != 1 || L.cols != r.msgs || L.weights[0] != 0) return fail(LOLA_E_PARAM, "combine shifts: 1 x messages, first 0");
    for (uint32_t m = 1; m < r.msgs; ++m) {
      if (L.weights[m] <= 0 || L.weights[m] >= (int64_t)h) return fail(LOLA_E_PARAM, "combine shifts must be in (0, n/2)");
      shift[m] = (uint64_t)L.weights[m];
    }
  } else {
    for (uint32_t m = 0; m < r.msgs; ++m) shift[m] = (uint64_t)m * L.stride;
  }
  Repr out = r;
  out.msgs = 1;
  std::set<uint32_t> used;
  for (auto& p : out.pos) {
    const uint64_t slot = (uint64_t)p.second + shift[p.first];
    if (p.second >= h || slot >= h) return fail(LOLA_E_PARAM, "combine would wrap a slot row");
    if (!used.insert((uint32_t)slot).second) return fail(LOLA_E_PARAM, "combine positions collide");
    p = {0, (uint32_t)slot};
  }
  if (r.msgs > 1) {
    const uint32_t k = r.msgs - 1;
    const int tmp = b.vreg(k);
    std::vector<int32_t> st;
    for (uint32_t m = 1; m <= k; ++m) st.push_back((int32_t)shift[m]);
    Op ro;
    b.rot(tmp, r.reg, -1, k, st);
    b.net->ops.back().src_off = 1;
    Op so;
    so.kind = OP_SUM;
    so.dst = b.vreg(1);
    so.src = tmp;
    so.msgs = k;
    so.aux = r.reg;
    so.aux_off = 0;
    b.net->ops.push_back(so);
    out.reg = so.dst;
  }
  r = out;
  return LOLA_OK;
}

// Combine k dense messages into one with element e at slot T[e], over both
// slot rows (Sec. 6.2: 83 maps of 196 values, more than one row holds).
// Each message's elements are grouped by the in-row right shift and by
// whether they change row; a message with several groups is masked per
// group (one ct x plaintext each); shifted groups rotate in waves of
// consecutive messages; the groups that change row are summed and
// row-swapped once, fused with the final addition.  Messages must hold
// zeros outside their elements' slots.
static int layer_place(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n, h = n / 2;
  if (r.kind != LOLA_REPR_DENSE && r.kind != LOLA_REPR_INTERLEAVED)
    return fail(LOLA_E_REPR, "place needs dense messages");
  const size_t E = r.pos.size();
  if (!L.weights || (size_t)L.rows * L.cols != E) return fail(LOLA_E_PARAM, "place needs one target slot per element");
  std::set<uint32_t> used;
  std::map<uint32_t, std::map<std::pair<int, uint32_t>, std::vector<uint32_t>>> groups;
  for (size_t e = 0; e < E; ++e) {
    const int64_t t = L.weights[e];
    if (t < 0 || t >= (int64_t)n) return fail(LOLA_E_PARAM, "place target out of range");
    if (!used.insert((uint32_t)t).second) return fail(LOLA_E_PARAM, "place targets collide");
    const uint32_t m = r.pos[e].first, s = r.pos[e].second;
    const uint32_t k = ((uint32_t)t % h + h - s % h) % h;
    const int swap = (s / h) != ((uint32_t)t / h) ? 1 : 0;
    groups[m][{swap, k}].push_back((uint32_t)e);
  }
  struct Term {
    int reg;
    uint32_t off;
    uint32_t k;
    int swap;
  };
  std::vector<Term> terms;
  for (auto& mg : groups) {
    const uint32_t m = mg.first;
    for (auto& g : mg.second) {
      Term tm{r.reg, m, g.first.second, g.first.first};
      if (mg.second.size() > 1) {
        std::vector<std::vector<int64_t>> M(1, std::vector<int64_t>(n, 0));
        for (uint32_t e : g.second) M[0][r.pos[e].second] = 1;
        Op mp;
        mp.kind = OP_MULPT;
        mp.src = r.reg;
        mp.src_off = m;
        mp.src_stride = 1;
        mp.dst = b.vreg(1);
        mp.msgs = 1;
        mp.pt_first = b.add_plaintexts(M);
        b.net->ops.push_back(mp);
        tm.reg = mp.dst;
        tm.off = 0;
      }
      terms.push_back(tm);
    }
  }
  // rotation waves over runs of consecutive source messages
  for (size_t i = 0; i < terms.size();) {
    if (terms[i].k == 0) {
      ++i;
      continue;
    }
    size_t j = i + 1;
    while (j < terms.size() && terms[j].k != 0 && terms[j].reg == terms[i].reg &&
           terms[j].off == terms[i].off + (uint32_t)(j - i))
      ++j;
    const uint32_t cnt = (uint32_t)(j - i);
    const int dst = b.vreg(cnt);
    std::vector<int32_t> st;
    for (size_t x = i; x < j; ++x) st.push_back((int32_t)terms[x].k);
    b.rot(dst, terms[i].reg, -1, cnt, st);
    b.net->ops.back().src_off = terms[i].off;
    for (size_t x = i; x < j; ++x) {
      terms[x].reg = dst;
      terms[x].off = (uint32_t)(x - i);
    }
    i = j;
  }
  // sums per row class, runs of consecutive messages per OP_SUM
  int acc[2] = {-1, -1};
  uint32_t acc_off[2] = {0, 0};
  for (int cls = 0; cls < 2; ++cls) {
    std::vector<Term> ts;
    for (auto& tm : terms)
      if (tm.swap == cls) ts.push_back(tm);
    for (size_t i = 0; i < ts.size();) {
      size_t j = i + 1;
      while (j < ts.size() && ts[j].reg == ts[i].reg && ts[j].off == ts[i].off + (uint32_t)(j - i)) ++j;
      if (acc[cls] < 0 && j - i == 1) {
        acc[cls] = ts[i].reg;                 // a lone first term is the accumulator as it is
        acc_off[cls] = ts[i].off;
      } else {
        Op so;
        so.kind = OP_SUM;
        so.dst = b.vreg(1);
        so.src = ts[i].reg;
        so.src_off = ts[i].off;
        so.msgs = (uint32_t)(j - i);
        so.aux = acc[cls];
        so.aux_off = acc_off[cls];
        b.net->ops.push_back(so);
        acc[cls] = so.dst;
        acc_off[cls] = 0;
      }
      i = j;
    }
  }
  Repr out;
  out.kind = r.kind;
  out.msgs = 1;
  if (acc[1] >= 0) {
    const int dst = b.vreg(1);
    b.rot(dst, acc[1], acc[0], 1, std::vector<int32_t>(1, 0));
    b.net->ops.back().src_off = acc_off[1];
    b.net->ops.back().aux_off = acc_off[0];
    out.reg = dst;
  } else if (acc_off[0] != 0) {
    Op so;                                    // move the lone term into a register of its own
    so.kind = OP_SUM;
    so.dst = b.vreg(1);
    so.src = acc[0];
    so.src_off = acc_off[0];
    so.msgs = 1;
    b.net->ops.push_back(so);
    out.reg = so.dst;
  } else {
    out.reg = acc[0];
  }
  for (size_t e = 0; e < E; ++e) out.pos.push_back({0, (uint32_t)L.weights[e]});
  r = out;
  return LOLA_OK;
}

static int layer_square(Builder& b, const lola_layer&, Repr& r) {
  Op o;
  o.kind = OP_SQUARE;
  o.src = r.reg;
  o.dst = b.vreg(r.msgs);
  o.msgs = r.msgs;
  b.net->ops.push_back(o);
  b.net->needs_relin = true;
  r.reg = o.dst;
  return LOLA_OK;
}

// Modulus switching to the first L.d primes of Q (not in the paper; every
// slot keeps its value): later layers run on fewer primes.
static int layer_mod_switch(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t Lv = L.d;
  if (Lv < 1 || Lv > b.level) return fail(LOLA_E_PARAM, "mod switch: level must be in [1, current level]");
  if (Lv == b.level) return LOLA_OK;
  Ctx* lc = nullptr;
  TRY(ctx_level(b.c, Lv, &lc));
  b.net->lctx[Lv] = lc;
  Op o;
  o.kind = OP_MODSWITCH;
  o.src = r.reg;
  o.msgs = r.msgs;
  o.level = b.level;
  o.level_to = Lv;
  b.level = Lv;
  b.lc = lc;
  o.dst = b.vreg(r.msgs);
  b.net->ops.push_back(o);
  r.reg = o.dst;
  return LOLA_OK;
}

static int layer_stack(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n, h = n / 2, s = 1u << L.d;
  if (r.msgs != 1 || (r.kind != LOLA_REPR_DENSE && r.kind != LOLA_REPR_INTERLEAVED))
    return fail(LOLA_E_REPR, "stack needs one dense message");
  if (L.d > 14 || L.copies == 0 || (L.copies & (L.copies - 1)) || (uint64_t)L.copies * s > n)
    return fail(LOLA_E_PARAM, "stack: copies must be a power of two with copies * 2^d <= n");
  for (auto& p : r.pos)
    if (p.second >= s) return fail(LOLA_E_PARAM, "stack: vector must fit in one block of 2^d slots");
  const uint32_t per_row = std::min<uint32_t>(L.copies, std::max<uint32_t>(1, h / s));
  std::vector<int32_t> shifts;
  for (uint32_t sh = s; sh < per_row * s; sh *= 2) shifts.push_back((int32_t)sh);
  if (L.copies > per_row) shifts.push_back(0);   // row swap
  r.reg = b.rotate_and_sum(r.reg, 1, shifts, L.hoist);
  r.kind = LOLA_REPR_STACKED;
  r.block = s;
  r.copies = L.copies;
  return LOLA_OK;
}

static uint32_t stacked_out_slot(uint32_t n, uint32_t s, uint32_t blk, uint32_t rnd) {
  const uint32_t h = n / 2, base = blk * s + s - 1;
  return (base / h) * h + (base % h + rnd) % h;
}

static int layer_stacked_rowmajor(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n;
  if (r.kind != LOLA_REPR_STACKED || r.msgs != 1) return fail(LOLA_E_REPR, "stacked row-major needs a stacked vector");
  const uint32_t s = 1u << L.d;
  if (s != r.block || L.copies != r.copies) return fail(LOLA_E_REPR, "stacked layout (d, copies) mismatch");
  if (!L.weights || L.cols != r.pos.size() || L.rows == 0) return fail(LOLA_E_PARAM, "weights must be rows x vector length");
  const uint32_t rows = L.rows, c = L.copies;
  const uint32_t R = (rows + c - 1) / c;
  if (R > s) return fail(LOLA_E_PARAM, "too many rounds for the block size");
  std::vector<std::vector<int64_t>> P(R, std::vector<int64_t>(n, 0));
  for (uint32_t rd = 0; rd < R; ++rd)
    for (uint32_t blk = 0; blk < c; ++blk) {
      const uint32_t row = rd * c + blk;
      if (row >= rows) continue;
      for (uint32_t i = 0; i < L.cols; ++i) P[rd][(size_t)blk * s + r.pos[i].second] = L.weights[(size_t)row * L.cols + i];
    }
  Op mp;
  mp.kind = OP_MULPT;
  mp.src = r.reg;
  mp.src_stride = 0;
  mp.dst = b.vreg(R);
  mp.msgs = R;
  mp.pt_first = b.add_plaintexts(P);
  b.net->ops.push_back(mp);
  std::vector<int32_t> shifts;
  for (uint32_t j = 0; j < L.d; ++j) shifts.push_back((int32_t)(1u << j));
  int y = b.rotate_and_sum(mp.dst, R, shifts, L.hoist);
  Repr out;
  out.kind = LOLA_REPR_INTERLEAVED;
  out.msgs = 1;
  if (R == 1) {
    out.reg = y;
    for (uint32_t row = 0; row < rows; ++row) out.pos.push_back({0, stacked_out_slot(n, s, row, 0)});
    r = out;
    return LOLA_OK;
  }
  // mask each round's block ends, rotate round rd right by rd, add
  std::vector<std::vector<int64_t>> M(R, std::vector<int64_t>(n, 0));
  for (uint32_t rd = 0; rd < R; ++rd)
    for (uint32_t blk = 0; blk < c; ++blk)
      if (rd * c + blk < rows) M[rd][(size_t)blk * s + s - 1] = 1;
  Op mk;
  mk.kind = OP_MULPT;
  mk.src = y;
  mk.src_stride = 1;
  mk.dst = b.vreg(R);
  mk.msgs = R;
  mk.pt_first = b.add_plaintexts(M);
  b.net->ops.push_back(mk);
  const int tmp = b.vreg(R - 1);
  std::vector<int32_t> st;
  for (uint32_t rd = 1; rd < R; ++rd) st.push_back((int32_t)rd);
  b.rot(tmp, mk.dst, -1, R - 1, st);
  b.net->ops.back().src_off = 1;
  Op so;
  so.kind = OP_SUM;
  so.dst = b.vreg(1);
  so.src = tmp;
  so.msgs = R - 1;
  so.aux = mk.dst;
  so.aux_off = 0;
  b.net->ops.push_back(so);
  out.reg = so.dst;
  for (uint32_t o = 0; o < rows; ++o) out.pos.push_back({0, stacked_out_slot(n, s, o % c, o / c)});
  r = out;
  return LOLA_OK;
}

static int layer_rowmajor_sparse(Builder& b, const lola_layer& L, Repr& r, bool dense_only) {
  const uint32_t n = b.c->n;
  if (r.msgs != 1) return fail(LOLA_E_REPR, "row-major product needs one message");
  if (dense_only && r.kind != LOLA_REPR_DENSE) return fail(LOLA_E_REPR, "dense row-major needs a dense vector");
  if (!dense_only && r.kind != LOLA_REPR_INTERLEAVED && r.kind != LOLA_REPR_DENSE)
    return fail(LOLA_E_REPR, "interleaved row-major needs an interleaved vector");
  if (!L.weights || L.cols != r.pos.size() || L.rows == 0) return fail(LOLA_E_PARAM, "weights must be rows x vector length");
  const uint32_t rows = L.rows;
  std::vector<std::vector<int64_t>> V(rows, std::vector<int64_t>(n, 0));
  for (uint32_t o = 0; o < rows; ++o)
    for (uint32_t i = 0; i < L.cols; ++i) V[o][r.pos[i].second] = L.weights[(size_t)o * L.cols + i];
  Op mp;
  mp.kind = OP_MULPT;
  mp.src = r.reg;
  mp.src_stride = 0;
  mp.dst = b.vreg(rows);
  mp.msgs = rows;
  mp.pt_first = b.add_plaintexts(V);
  b.net->ops.push_back(mp);
  std::vector<int32_t> shifts;
  for (uint32_t sh = 1; sh < n / 2; sh *= 2) shifts.push_back((int32_t)sh);
  shifts.push_back(0);
  Repr out;
  out.kind = LOLA_REPR_SPARSE;
  out.msgs = rows;
  out.reg = b.rotate_and_sum(mp.dst, rows, shifts, L.hoist);
  for (uint32_t o = 0; o < rows; ++o) out.pos.push_back({o, 0});
  r = out;
  return LOLA_OK;
}

// Rotate-and-sum steps that add every occupied slot of a message into one
// slot, and that slot (the support-summed row-major product).  When the
// occupied slots of each row lie in one cyclic run of 2^k slots modulo a
// period 2^p, the right rotations 1 .. 2^(k-1) (the run), then 2^p .. n/4
// (the period), then the row swap if both rows are occupied add each
// occupied slot exactly once into one slot; the (p, k) with the fewest steps
// is taken, the smallest p on ties.  The full support (p = 0) gives the
// interleaved row-major product's 1, 2, ..., n/4 and the row swap.  The
// result slot is the smallest slot whose occupancy count after the steps
// equals the number of occupied slots.
static void support_sum_shifts(const std::vector<uint32_t>& slots, uint32_t n, std::vector<int32_t>* shifts,
                               uint32_t* result_slot) {
  const uint32_t h = n / 2;
  uint32_t logh = 0;
  while ((1u << logh) < h) ++logh;
  std::set<uint32_t> rows, cols;
  for (uint32_t s : slots) {
    rows.insert(s / h);
    cols.insert(s % h);
  }
  int best = -1;
  uint32_t best_p = 0, best_k = 0;
  for (uint32_t lp = 0; lp <= logh; ++lp) {
    const uint32_t per = 1u << lp;
    std::set<uint32_t> res;
    for (uint32_t c : cols) res.insert(c % per);
    for (uint32_t k = 0; k <= lp; ++k) {
      const uint32_t run = 1u << k;
      bool ok = false;
      for (uint32_t o : res) {
        bool all = true;
        for (uint32_t c : res)
          if ((c + per - o) % per >= run) {
            all = false;
            break;
          }
        if (all) {
          ok = true;
          break;
        }
      }
      if (!ok) continue;
      const int cnt = (int)(k + (logh - lp) + (rows.size() > 1 ? 1 : 0));
      if (best < 0 || cnt < best) {
        best = cnt;
        best_p = lp;
        best_k = k;
      }
      break;
    }
  }
  shifts->clear();
  for (uint32_t j = 0; j < best_k; ++j) shifts->push_back((int32_t)(1u << j));
  for (uint32_t j = best_p; j < logh; ++j) shifts->push_back((int32_t)(1u << j));
  if (rows.size() > 1) shifts->push_back(0);
  std::vector<uint32_t> cnt(n, 0), nxt(n);
  for (uint32_t s : slots) cnt[s] = 1;
  for (int32_t sh : *shifts) {
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t r = i / h, c = i % h;
      const uint32_t src = sh == 0 ? (r ^ 1) * h + c : r * h + (c + h - (uint32_t)sh) % h;
      nxt[i] = cnt[i] + cnt[src];
    }
    cnt.swap(nxt);
  }
  const uint32_t want = (uint32_t)std::set<uint32_t>(slots.begin(), slots.end()).size();
  *result_slot = 0;
  for (uint32_t i = 0; i < n; ++i)
    if (cnt[i] == want) {
      *result_slot = i;
      break;
    }
}

// Interleaved vector - row major with each dot product summed over the
// vector's occupied slots only (support_sum_shifts): the products of
// layer_rowmajor_sparse, the support's rotate-and-sum, output o = message o
// at the one slot holding the whole sum.
static int layer_rowmajor_support(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n;
  if (r.msgs != 1 || (r.kind != LOLA_REPR_INTERLEAVED && r.kind != LOLA_REPR_DENSE))
    return fail(LOLA_E_REPR, "support-summed row-major product needs one interleaved or dense message");
  if (!L.weights || L.cols != r.pos.size() || L.rows == 0) return fail(LOLA_E_PARAM, "weights must be rows x vector length");
  const uint32_t rows = L.rows;
  std::vector<std::vector<int64_t>> V(rows, std::vector<int64_t>(n, 0));
  std::vector<uint32_t> slots;
  for (auto& p : r.pos) slots.push_back(p.second);
  for (uint32_t o = 0; o < rows; ++o)
    for (uint32_t i = 0; i < L.cols; ++i) V[o][r.pos[i].second] = L.weights[(size_t)o * L.cols + i];
  Op mp;
  mp.kind = OP_MULPT;
  mp.src = r.reg;
  mp.src_stride = 0;
  mp.dst = b.vreg(rows);
  mp.msgs = rows;
  mp.pt_first = b.add_plaintexts(V);
  b.net->ops.push_back(mp);
  std::vector<int32_t> shifts;
  uint32_t slot = 0;
  support_sum_shifts(slots, n, &shifts, &slot);
  Repr out;
  out.kind = LOLA_REPR_DENSE;
  out.msgs = rows;
  out.reg = b.rotate_and_sum(mp.dst, rows, shifts, L.hoist);
  for (uint32_t o = 0; o < rows; ++o) out.pos.push_back({o, slot});
  r = out;
  return LOLA_OK;
}

// Sparse vector - column major (Sec. 4.2.2): W v = sum_i v_i c^i.  Message i
// holds v_i in every slot; multiply it by column i of W laid out densely
// (slot o = W[o][i]) and add the products.  No rotations; dense result.
static int layer_sparse_colmajor(Builder& b, const lola_layer& L, Repr& r) {
  const uint32_t n = b.c->n;
  if (r.kind != LOLA_REPR_SPARSE) return fail(LOLA_E_REPR, "column-major product needs a sparse vector");
  if (!L.weights || L.cols != r.msgs || L.rows == 0 || L.rows > n)
    return fail(LOLA_E_PARAM, "weights must be rows x (number of sparse messages), rows <= n");
  const uint32_t k = L.cols, rows = L.rows;
  std::vector<std::vector<int64_t>> Cc(k, std::vector<int64_t>(n, 0));
  for (uint32_t i = 0; i < k; ++i)
    for (uint32_t o = 0; o < rows; ++o) Cc[i][o] = L.weights[(size_t)o * k + i];
  Op mp;
  mp.kind = OP_MULPT;
  mp.src = r.reg;
  mp.src_stride = 1;
  mp.dst = b.vreg(k);
  mp.msgs = k;
  mp.pt_first = b.add_plaintexts(Cc);
  b.net->ops.push_back(mp);
  Repr out;
  out.kind = LOLA_REPR_DENSE;
  out.msgs = 1;
  out.reg = mp.dst;
  if (k > 1) {
    Op so;
    so.kind = OP_SUM;
    so.dst = b.vreg(1);
    so.src = mp.dst;
    so.msgs = k;
    b.net->ops.push_back(so);
    out.reg = so.dst;
  }
  for (uint32_t o = 0; o < rows; ++o) out.pos.push_back({0, o});
  r = out;
  return LOLA_OK;
}

Net::~Net() {}

int net_create(Ctx* c, const lola_input* in, const lola_layer* layers, size_t n_layers, Net** out) {
  if (!in || (!layers && n_layers) || !out) return fail(LOLA_E_PARAM, "null argument");
  *out = nullptr;
  std::unique_ptr<Net> net(new Net());
  net->ctx = c;
  Builder b;
  b.c = c;
  b.net = net.get();
  b.level = c->L;
  b.lc = c;
  net->lctx[c->L] = c;
  Repr r;
  r.kind = in->repr;
  r.msgs = in->n_msgs;
  if (in->n_msgs == 0 || in->n_elems == 0) return fail(LOLA_E_PARAM, "empty input");
  for (uint32_t i = 0; i < in->n_elems; ++i) {
    const uint32_t slot = in->slot ? in->slot[i] : i;
    if (slot >= c->n) return fail(LOLA_E_PARAM, "input slot out of range");
    r.pos.push_back({0, slot});
  }
  if (in->repr == LOLA_REPR_STACKED) {
    r.block = 1u << in->d;
    r.copies = in->copies;
  }
  r.reg = b.vreg(in->n_msgs);
  net->in_reg = r.reg;
  net->n_in = in->n_msgs;
  for (size_t li = 0; li < n_layers; ++li) {
    const lola_layer& L = layers[li];
    if (L.in_repr && L.in_repr != r.kind)
      return fail(LOLA_E_REPR, "layer " + std::to_string(li) + ": input representation mismatch");
    const size_t op0 = net->ops.size();
    int rc;
    switch (L.op) {
      case LOLA_LAYER_CONV_ROWMAJOR: rc = layer_conv(b, L, r); break;
      case LOLA_LAYER_COMBINE: rc = layer_combine(b, L, r); break;
      case LOLA_LAYER_MASKED_SHIFTS: rc = layer_masked_shifts(b, L, r); break;
      case LOLA_LAYER_PLACE: rc = layer_place(b, L, r); break;
      case LOLA_LAYER_SQUARE: rc = layer_square(b, L, r); break;
      case LOLA_LAYER_STACK: rc = layer_stack(b, L, r); break;
      case LOLA_LAYER_STACKED_ROWMAJOR: rc = layer_stacked_rowmajor(b, L, r); break;
      case LOLA_LAYER_INTERLEAVED_ROWMAJOR: rc = layer_rowmajor_sparse(b, L, r, false); break;
      case LOLA_LAYER_DENSE_ROWMAJOR: rc = layer_rowmajor_sparse(b, L, r, true); break;
      case LOLA_LAYER_SPARSE_COLMAJOR: rc = layer_sparse_colmajor(b, L, r); break;
      case LOLA_LAYER_MOD_SWITCH: rc = layer_mod_switch(b, L, r); break;
      case LOLA_LAYER_INTERLEAVED_ROWMAJOR_SUPPORT: rc = layer_rowmajor_support(b, L, r); break;
      default: return fail(LOLA_E_PARAM, "unknown layer op");
    }
    if (rc != LOLA_OK) return rc;
    for (size_t i = op0; i < net->ops.size(); ++i)
      if (!net->ops[i].level) net->ops[i].level = b.level;
    if (L.out_repr && L.out_repr != r.kind)
      return fail(LOLA_E_REPR, "layer " + std::to_string(li) + ": output representation mismatch");
  }
  net->out_reg = r.reg;
  net->out_level = b.level;
  net->n_out = r.msgs;
  for (auto& p : r.pos) {
    net->out_msg.push_back(p.first);
    net->out_slot.push_back(p.second);
  }
  net->steps_needed.assign(b.steps.begin(), b.steps.end());
  // encode plaintexts for every t_i, per level: blocks [pt][kt][level][n]
  const size_t kt = c->kt, n = c->n;
  for (auto& lp : b.pts) {
    const uint32_t Lv = lp.first;
    const auto& pts = lp.second;
    Ctx* lc = net->lctx.at(Lv);
    DevBuf& buf = net->pt[Lv];
    TRY(buf.alloc(pts.size() * kt * Lv * n * 8));
    std::vector<int64_t> slots;
    std::vector<uint32_t> tidx;
    const size_t chunk = 64;
    for (size_t p0 = 0; p0 < pts.size(); p0 += chunk) {
      const size_t p1 = std::min(pts.size(), p0 + chunk);
      slots.clear();
      tidx.clear();
      for (size_t p = p0; p < p1; ++p)
        for (size_t ti = 0; ti < kt; ++ti) {
          slots.insert(slots.end(), pts[p].begin(), pts[p].end());
          tidx.push_back((uint32_t)ti);
        }
      TRY(encode_plaintexts(lc, slots.data(), tidx.data(), (p1 - p0) * kt, buf.u64() + p0 * kt * Lv * n, nullptr));
    }
  }
  if (!b.w.empty()) {
    TRY(net->w.alloc(b.w.size() * 8));
    TRY(net->ws.alloc(b.ws.size() * 8));
    LOLA_CUDA_TRY(cudaMemcpy(net->w.p, b.w.data(), b.w.size() * 8, cudaMemcpyHostToDevice));
    LOLA_CUDA_TRY(cudaMemcpy(net->ws.p, b.ws.data(), b.ws.size() * 8, cudaMemcpyHostToDevice));
  }
  *out = net.release();
  return LOLA_OK;
}

// ------------------------------------------------------------------- executor
// largest rotation wave (ciphertexts) per launch sequence; at n = 16384, L = 6
// its key-switch scratch is about 7.5 GB
static constexpr uint32_t kMaxRotCts = 1024;

struct Executor {
  uint32_t B = 0;
  std::vector<DevBuf> phys;            // physical register buffers
  std::vector<int> vmap;               // virtual -> physical
  DevBuf scratch;
  DevBuf tid_pattern;                  // i % kt
  const KeySet* keys = nullptr;        // key set the device tables were built for
  std::vector<DevBuf> op_gal, op_keys; // per-op per-message tables (non-uniform rotations)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  ~Executor() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

static int build_executor(Ctx* c, Net* net, uint32_t B, Executor* ex) {
  ex->B = B;
  const size_t kt = c->kt, ctw = c->ct_words();
  const size_t msg_words = (size_t)B * kt * ctw;
  // liveness: last op index using each vreg
  const int nv = (int)net->vreg_msgs.size();
  std::vector<int> last(nv, -1), first(nv, (int)net->ops.size());
  first[net->in_reg] = -1;
  for (int i = 0; i < (int)net->ops.size(); ++i) {
    const Op& o = net->ops[i];
    for (int v : {o.src, o.aux})
      if (v >= 0) last[v] = std::max(last[v], i);
    if (o.dst >= 0) first[o.dst] = std::min(first[o.dst], i);
  }
  last[net->out_reg] = (int)net->ops.size();
  ex->vmap.assign(nv, -1);
  std::vector<uint32_t> phys_msgs;
  std::vector<int> phys_free_after;   // op index after which the buffer is free
  auto assign = [&](int v, int at) {
    int best = -1;
    for (int p = 0; p < (int)phys_msgs.size(); ++p)
      if (phys_free_after[p] < at && phys_msgs[p] >= net->vreg_msgs[v] &&
          (best < 0 || phys_msgs[p] < phys_msgs[best]))
        best = p;
    if (best < 0) {
      phys_msgs.push_back(net->vreg_msgs[v]);
      phys_free_after.push_back(0);
      best = (int)phys_msgs.size() - 1;
    }
    ex->vmap[v] = best;
    phys_free_after[best] = std::max(last[v], at);
  };
  assign(net->in_reg, -1);
  for (int i = 0; i < (int)net->ops.size(); ++i) {
    const int d = net->ops[i].dst;
    if (d >= 0 && ex->vmap[d] < 0) assign(d, i);
  }
  ex->phys.resize(phys_msgs.size());
  for (size_t p = 0; p < phys_msgs.size(); ++p) TRY(ex->phys[p].alloc(phys_msgs[p] * msg_words * 8));
  // scratch: largest op requirement (each at its level)
  size_t sw = 0, maxcnt = 1;
  for (const Op& o : net->ops) {
    const Ctx* lc = net->lctx.at(o.level);
    const size_t cnt = (size_t)o.msgs * B * kt;
    maxcnt = std::max(maxcnt, cnt);
    if (o.kind == OP_ROT || o.kind == OP_ROT_SUM) {
      const size_t per_msg = (size_t)B * kt;
      const size_t chunk_msgs = std::max<size_t>(1, kMaxRotCts / per_msg);
      const size_t mc = std::min<size_t>(o.msgs, chunk_msgs);
      sw = std::max(sw, o.kind == OP_ROT ? rotate_scratch_words(lc, mc * per_msg) + 2 * mc
                                         : rotate_sum_scratch_words(lc, mc * per_msg));
    }
    if (o.kind == OP_SQUARE) sw = std::max(sw, multiply_scratch_words(lc, cnt, true));
    if (o.kind == OP_ROT_HOISTED) sw = std::max(sw, rotate_hoisted_scratch_words(lc, (size_t)B * kt, o.msgs));
    if (o.kind == OP_MODSWITCH) sw = std::max(sw, mod_switch_scratch_words(c, cnt, o.level, o.level_to));
  }
  TRY(ex->scratch.alloc(sw * 8));
  std::vector<uint32_t> pat(maxcnt);
  for (size_t i = 0; i < maxcnt; ++i) pat[i] = (uint32_t)(i % kt);
  TRY(ex->tid_pattern.alloc(maxcnt * 4));
  LOLA_CUDA_TRY(cudaMemcpy(ex->tid_pattern.p, pat.data(), maxcnt * 4, cudaMemcpyHostToDevice));
  return LOLA_OK;
}

static int bind_keys(Ctx* c, Net* net, Executor* ex, const KeySet* ks) {
  if (ex->keys == ks) return LOLA_OK;
  if (net->needs_relin && !ks->ev->relin) return fail(LOLA_E_NOKEY, "network squares but no relinearisation key");
  ex->op_gal.clear();
  ex->op_keys.clear();
  ex->op_gal.resize(net->ops.size());
  ex->op_keys.resize(net->ops.size());
  for (size_t i = 0; i < net->ops.size(); ++i) {
    const Op& o = net->ops[i];
    if (o.kind != OP_ROT && o.kind != OP_ROT_HOISTED && o.kind != OP_ROT_SUM) continue;
    const size_t ne = o.kind == OP_ROT_SUM ? o.steps.size() : o.msgs;   // table entries
    std::vector<uint32_t> g(ne);
    std::vector<const uint64_t*> kp(ne);
    for (size_t m = 0; m < ne; ++m) {
      g[m] = galois_for_step(c->n, o.steps[m]);
      const SwitchKey* key = ks->galois_key(g[m]);
      if (!key) return fail(LOLA_E_NOKEY, "missing Galois key for rotation step " + std::to_string(o.steps[m]));
      kp[m] = key->buf.u64();
    }
    TRY(ex->op_gal[i].alloc(ne * 4));
    TRY(ex->op_keys[i].alloc(ne * 8));
    LOLA_CUDA_TRY(cudaMemcpy(ex->op_gal[i].p, g.data(), ne * 4, cudaMemcpyHostToDevice));
    LOLA_CUDA_TRY(cudaMemcpy(ex->op_keys[i].p, kp.data(), ne * 8, cudaMemcpyHostToDevice));
  }
  if (ex->graph) {
    cudaGraphExecDestroy(ex->graph);
    ex->graph = nullptr;
  }
  ex->keys = ks;
  return LOLA_OK;
}

static int run_ops(Ctx* root, Net* net, Executor* ex, const KeySet* ks, cudaStream_t s) {
  const size_t kt = root->kt;
  const uint32_t B = ex->B;
  // message m of register v: [request][t_i][2][level(v)][n] words at m * B kt 2 level n
  auto reg = [&](int v, uint32_t off) {
    return ex->phys[ex->vmap[v]].u64() + (size_t)off * B * kt * 2 * net->vreg_level[v] * root->n;
  };
  for (size_t i = 0; i < net->ops.size(); ++i) {
    const Op& o = net->ops[i];
    Ctx* c = net->lctx.at(o.level);
    const size_t msg_words = (size_t)B * kt * c->ct_words();
    const size_t cnt = (size_t)o.msgs * B * kt;
    switch (o.kind) {
      case OP_MAC:
        TRY(k::mac_scalar(c, reg(o.src, o.src_off), o.R, net->w.u64() + o.w_first, net->ws.u64() + o.w_first,
                          reg(o.dst, o.dst_off), o.msgs, B, s));
        break;
      case OP_ROT: {
        const bool uniform = std::all_of(o.steps.begin(), o.steps.end(), [&](int32_t x) { return x == o.steps[0]; });
        // waves larger than kMaxRotCts ciphertexts run in chunks of whole
        // messages, which bounds the key-switch scratch
        const uint32_t per_msg = (uint32_t)(B * kt);
        const uint32_t chunk = std::max<uint32_t>(1, kMaxRotCts / per_msg);
        for (uint32_t m0 = 0; m0 < o.msgs; m0 += chunk) {
          const uint32_t mc = std::min(chunk, o.msgs - m0);
          RotSpec rs;
          if (uniform) {
            rs.gal = galois_for_step(c->n, o.steps[0]);
            rs.key = ks->galois_key(rs.gal)->buf.u64();
          } else {
            rs.d_gal = (const uint32_t*)ex->op_gal[i].p + m0;
            rs.d_keys = (const uint64_t* const*)ex->op_keys[i].p + m0;
            rs.div = per_msg;
          }
          TRY(rotate(c, reg(o.src, o.src_off + m0), reg(o.dst, o.dst_off + m0),
                     o.aux >= 0 ? reg(o.aux, o.aux_off + m0) : nullptr, (size_t)mc * per_msg, rs, ex->scratch.u64(),
                     s));
        }
        break;
      }
      case OP_ROT_SUM: {
        const uint32_t per_msg = (uint32_t)(B * kt);
        const uint32_t chunk = std::max<uint32_t>(1, kMaxRotCts / per_msg);
        for (uint32_t m0 = 0; m0 < o.msgs; m0 += chunk) {
          const uint32_t mc = std::min(chunk, o.msgs - m0);
          // every ciphertext of the chunk uses the op's one list of steps
          TRY(rotate_sum(c, reg(o.src, o.src_off + m0), reg(o.dst, o.dst_off + m0), (size_t)mc * per_msg,
                         (uint32_t)o.steps.size(), (const uint32_t*)ex->op_gal[i].p,
                         (const uint64_t* const*)ex->op_keys[i].p, mc * per_msg, ex->scratch.u64(), s));
        }
        break;
      }
      case OP_ROT_HOISTED:
        TRY(rotate_hoisted(c, reg(o.src, o.src_off), reg(o.dst, o.dst_off), (size_t)B * kt, o.msgs,
                           (const uint32_t*)ex->op_gal[i].p, (const uint64_t* const*)ex->op_keys[i].p,
                           ex->scratch.u64(), s));
        break;
      case OP_SUM: {
        uint64_t* d = reg(o.dst, o.dst_off);
        const size_t per = (size_t)B * kt;
        if (o.aux < 0 && o.msgs == 1) {
          LOLA_CUDA_TRY(cudaMemcpyAsync(d, reg(o.src, o.src_off), msg_words * 8, cudaMemcpyDeviceToDevice, s));
        } else {
          // one launch for the whole sum (the messages of a register are contiguous)
          TRY(k::sum_msgs(c, reg(o.src, o.src_off), o.msgs, o.aux >= 0 ? reg(o.aux, o.aux_off) : nullptr, d, per, s));
        }
        break;
      }
      case OP_MULPT: {
        const uint64_t* pt = net->pt.at(o.level).u64() + o.pt_first * kt * c->L * c->n;
        // src_stride 0: one input message times every plaintext; 1: message m times plaintext m
        TRY(k::mul_plain_multi(c, reg(o.src, o.src_off), pt, reg(o.dst, o.dst_off), o.msgs, B, s, o.src_stride != 0));
        break;
      }
      case OP_SQUARE:
        TRY(multiply(c, reg(o.src, o.src_off), reg(o.src, o.src_off), reg(o.dst, o.dst_off), cnt,
                     (const uint32_t*)ex->tid_pattern.p, 1, ks->ev->relin->buf.u64(), ex->scratch.u64(), s));
        break;
      case OP_MODSWITCH:
        TRY(mod_switch(root, reg(o.src, o.src_off), reg(o.dst, o.dst_off), cnt, o.level, o.level_to,
                       ex->scratch.u64(), s));
        break;
    }
  }
  return LOLA_OK;
}

// request-major lola_ct layout [b][g][t] <-> register layout [g][b][t]
static int transpose_msgs(uint64_t* dst, const uint64_t* src, uint32_t G, uint32_t B, size_t blk_words, bool to_reg,
                          cudaStream_t s) {
  if (G == 1 || B == 1) {
    LOLA_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)G * B * blk_words * 8, cudaMemcpyDeviceToDevice, s));
    return LOLA_OK;
  }
  for (uint32_t g = 0; g < G; ++g) {
    const size_t bytes = blk_words * 8;
    if (to_reg) {
      LOLA_CUDA_TRY(cudaMemcpy2DAsync(dst + (size_t)g * B * blk_words, bytes, src + (size_t)g * blk_words,
                                      (size_t)G * bytes, bytes, B, cudaMemcpyDeviceToDevice, s));
    } else {
      LOLA_CUDA_TRY(cudaMemcpy2DAsync(dst + (size_t)g * blk_words, (size_t)G * bytes, src + (size_t)g * B * blk_words,
                                      bytes, bytes, B, cudaMemcpyDeviceToDevice, s));
    }
  }
  return LOLA_OK;
}

int net_eval(Ctx* c, const KeySet* ks, Net* net, const uint64_t* d_in, size_t in_msgs, uint64_t* d_out,
             size_t out_msgs, cudaStream_t s, bool use_graph) {
  if (in_msgs == 0 || in_msgs % net->n_in) return fail(LOLA_E_PARAM, "input message count is not a multiple of the network input");
  const uint32_t B = (uint32_t)(in_msgs / net->n_in);
  if (out_msgs != (size_t)B * net->n_out) return fail(LOLA_E_PARAM, "output ciphertext has the wrong message count");
  auto& slot = net->exec[B];
  if (!slot) {
    std::unique_ptr<Executor> ex(new Executor());
    TRY(build_executor(c, net, B, ex.get()));
    slot = std::move(ex);
  }
  Executor* ex = slot.get();
  TRY(bind_keys(c, net, ex, ks));
  const size_t blk = (size_t)c->kt * c->ct_words();
  const size_t blk_out = (size_t)c->kt * 2 * net->out_level * c->n;
  TRY(transpose_msgs(ex->phys[ex->vmap[net->in_reg]].u64(), d_in, net->n_in, B, blk, true, s));
  const bool profiling = c->root->prof.any();
  if (use_graph && !profiling) {
    if (!ex->graph) {
      if (!ex->cap_stream) LOLA_CUDA_TRY(cudaStreamCreateWithFlags(&ex->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      LOLA_CUDA_TRY(cudaStreamBeginCapture(ex->cap_stream, cudaStreamCaptureModeThreadLocal));
      int rc = run_ops(c, net, ex, ks, ex->cap_stream);
      cudaError_t e = cudaStreamEndCapture(ex->cap_stream, &g);
      if (rc != LOLA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ex->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        ex->graph = nullptr;
        return fail(LOLA_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    LOLA_CUDA_TRY(cudaGraphLaunch(ex->graph, s));
  } else {
    TRY(run_ops(c, net, ex, ks, s));
  }
  TRY(transpose_msgs(d_out, ex->phys[ex->vmap[net->out_reg]].u64(), net->n_out, B, blk_out, false, s));
  return LOLA_OK;
}

}  // namespace lola
