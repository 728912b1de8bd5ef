// Context: parameter validation, prime tables, NTT twiddles and the exact
// CRT / mixed-radix constants used by the basis conversions.
#include <string.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "kernels.h"

namespace lola {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
const char* last_error() { return g_last_error.c_str(); }

// -------------------------------------------------------------- host math
uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod_h(r, b, q);
    b = mulmod_h(b, b, q);
    e >>= 1;
  }
  return r;
}
uint64_t invmod_h(uint64_t a, uint64_t q) { return powmod_h(a % q, q - 2, q); }  // q prime
uint64_t shoup_h(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

bool is_prime_h(uint64_t x) {
  if (x < 2) return false;
  static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint64_t p : small)
    if (x % p == 0) return x == p;
  uint64_t d = x - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint64_t a : small) {  // deterministic for 64-bit inputs
    uint64_t y = powmod_h(a, d, x);
    if (y == 1 || y == x - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      y = mulmod_h(y, y, x);
      if (y == x - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

// smallest primitive 2n-th root of unity: find one root x (x^n = -1), then
// the minimum over its odd powers (the primitive 2n-th roots).
uint64_t smallest_root_2n(uint64_t q, uint32_t n) {
  uint64_t x = 0;
  for (uint64_t g = 2; g < q; ++g) {
    x = powmod_h(g, (q - 1) / (2 * (uint64_t)n), q);
    if (powmod_h(x, n, q) == q - 1) break;
  }
  uint64_t best = x, x2 = mulmod_h(x, x, q), cur = x;
  for (uint32_t i = 1; i < n; ++i) {
    cur = mulmod_h(cur, x2, q);
    best = std::min(best, cur);
  }
  return best;
}

static uint32_t brev_h(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

uint32_t galois_for_step(uint32_t n, int32_t step) {
  const uint64_t two_n = 2ull * n;
  if (step == 0) return (uint32_t)(two_n - 1);
  const uint32_t e = (uint32_t)(n / 2 - (uint32_t)step);
  return (uint32_t)powmod_h(3, e, two_n);
}

// --------------------------------------------------------------- DevBuf
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    if (p) cudaFree(p);
    p = o.p;
    bytes = o.bytes;
    o.p = nullptr;
    o.bytes = 0;
  }
  return *this;
}
DevBuf::~DevBuf() {
  if (p) cudaFree(p);
}
int DevBuf::alloc(size_t nbytes) {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
  if (nbytes == 0) return LOLA_OK;
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(LOLA_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  bytes = nbytes;
  return LOLA_OK;
}

// ------------------------------------------------------------- profiling
const char* kernel_name(int id) {
  static const char* names[KI_COUNT] = {
      "ntt_fwd", "ntt_inv", "ntt_fwd_signed", "encode_lift", "slots_to_coeff", "coeff_to_slots", "enc_msg",
      "ks_decompose", "ks_modup", "ks_intt_p", "ks_moddown", "ks_ip",
      "add", "mul_plain", "mac_scalar", "tensor", "lift_q_to_b", "scale_round", "decrypt_round", "misc",
      "mod_switch", "ks_ip_sum"};
  return (id >= 0 && id < KI_COUNT) ? names[id] : "?";
}

void prof_begin(Ctx* c, int kind, cudaStream_t s, cudaEvent_t* ev) {
  c = c->root;
  if (!c->prof.on[kind]) return;
  if (c->prof.pool.empty()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    c->prof.pool.push_back({a, b});
  }
  auto pr = c->prof.pool.back();
  c->prof.pool.pop_back();
  ev[0] = pr.first;
  ev[1] = pr.second;
  cudaEventRecord(ev[0], s);
}
void prof_end(Ctx* c, int kind, cudaStream_t s, cudaEvent_t* ev, uint64_t units) {
  if (!ev[0]) return;
  c = c->root;
  cudaEventRecord(ev[1], s);
  c->prof.pending[kind].push_back({ev[0], ev[1], units});
}

static void prof_collect(Ctx* c, int kind) {
  for (auto& pr : c->prof.pending[kind]) {
    cudaEventSynchronize(pr.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, pr.a, pr.b);
    c->prof.ms[kind] += ms;
    c->prof.launches[kind] += 1;
    c->prof.units[kind] += pr.units;
    c->prof.pool.push_back({pr.a, pr.b});
  }
  c->prof.pending[kind].clear();
}

// ----------------------------------------------------------- context build
static void mrc_table(const std::vector<uint64_t>& basis, MrcDev& T) {
  const int k = (int)basis.size();
  memset(&T, 0, sizeof(T));
  T.k = k;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < i; ++j) {
      T.inv[i][j] = invmod_h(basis[j] % basis[i], basis[i]);
      T.inv_s[i][j] = shoup_h(T.inv[i][j], basis[i]);
    }
  // digits of H = (prod b - 1) / 2: residues H mod b_i = (b_i - 1) / 2, then Garner
  std::vector<uint64_t> v(k);
  for (int i = 0; i < k; ++i) {
    uint64_t u = (basis[i] - 1) / 2;
    for (int j = 0; j < i; ++j) {
      const uint64_t vj = v[j] % basis[i];
      u = mulmod_h((u + basis[i] - vj) % basis[i], T.inv[i][j], basis[i]);
    }
    v[i] = u;
    T.half[i] = u;
  }
}

// product of the first k primes of `basis` mod m
static uint64_t prefix_prod_mod(const std::vector<uint64_t>& basis, int k, uint64_t m) {
  uint64_t r = 1 % m;
  for (int i = 0; i < k; ++i) r = mulmod_h(r, basis[i] % m, m);
  return r;
}

static int build_ctx(Ctx* c, const lola_params* p) {
  c->n = p->n;
  c->logn = 0;
  while ((1u << c->logn) < p->n) ++c->logn;
  c->L = p->L;
  c->K = p->K;
  c->kt = p->k_t;
  c->alpha = p->alpha ? p->alpha : 1;
  if ((1u << c->logn) != p->n || c->logn < 4 || c->logn > 14) return fail(LOLA_E_PARAM, "n must be a power of two in [16, 16384]");
  if (p->L < 1 || p->L > MAXL) return fail(LOLA_E_PARAM, "L out of range");
  if (p->K > 2) return fail(LOLA_E_PARAM, "K must be 0, 1 or 2");
  if (c->alpha > 2) return fail(LOLA_E_PARAM, "alpha must be 0, 1 or 2");
  if (c->alpha > 1 && p->K == 0) return fail(LOLA_E_PARAM, "digits of several primes need a special prime (K > 0)");
  c->dnum = (c->L + c->alpha - 1) / c->alpha;
  if (p->k_t < 1 || p->k_t > MAXT) return fail(LOLA_E_PARAM, "k_t out of range");
  if (!p->q || !p->t) return fail(LOLA_E_PARAM, "null prime list");
  const uint64_t two_n = 2ull * p->n;
  std::vector<uint64_t> qp(p->q, p->q + p->L + p->K), ts(p->t, p->t + p->k_t);
  // the forward transforms' lazy bound (values below 8q + 2^32) needs q < 2^61 - 2^30
  const uint64_t qmax = (1ull << 61) - (1ull << 30);
  for (uint64_t q : qp)
    if (q >= qmax || q % two_n != 1 || !is_prime_h(q))
      return fail(LOLA_E_PARAM, "ciphertext prime must be prime, = 1 mod 2n, < 2^61 - 2^30");
  for (uint64_t t : ts)
    if (t >= (1ull << 31) || t % two_n != 1 || !is_prime_h(t)) return fail(LOLA_E_PARAM, "plaintext modulus must be prime, = 1 mod 2n, < 2^31");
  std::vector<uint64_t> all = qp;
  all.insert(all.end(), ts.begin(), ts.end());
  std::sort(all.begin(), all.end());
  if (std::adjacent_find(all.begin(), all.end()) != all.end()) return fail(LOLA_E_PARAM, "primes must be distinct");

  // auxiliary basis for exact ct x ct scaling: prod B > t n Q * 8
  double need = std::log2((double)p->n) + 3.0;
  for (uint32_t i = 0; i < p->L; ++i) need += std::log2((double)qp[i]);
  double tmax = 0;
  for (uint64_t t : ts) tmax = std::max(tmax, std::log2((double)t));
  need += tmax;
  std::vector<uint64_t> aux;
  double have = 0;
  for (uint64_t x = (qmax - 1) / two_n * two_n + 1; have < need; x -= two_n) {
    if (x >= qmax || !is_prime_h(x)) continue;
    if (std::find(qp.begin(), qp.end(), x) != qp.end()) continue;
    aux.push_back(x);
    have += std::log2((double)x);
  }
  if (aux.size() > MAXB) return fail(LOLA_E_PARAM, "auxiliary basis too large");
  c->M = (uint32_t)aux.size();
  c->primes = qp;
  c->primes.insert(c->primes.end(), aux.begin(), aux.end());
  c->primes.insert(c->primes.end(), ts.begin(), ts.end());
  const uint32_t np = (uint32_t)c->primes.size();
  if (np > MAXP) return fail(LOLA_E_PARAM, "too many primes");

  CtxDev& H = c->host;
  memset(&H, 0, sizeof(H));
  H.n = c->n;
  H.logn = c->logn;
  H.L = c->L;
  H.K = c->K;
  H.M = c->M;
  H.kt = c->kt;
  H.np = np;
  H.iP = c->iP();
  {
    const uint64_t qlo = *std::min_element(qp.begin(), qp.end()), qhi = *std::max_element(qp.begin(), qp.end());
    H.modup_raw = qhi / 8 < qlo ? 1u : 0u;
  }
  H.iB = c->iB();
  H.iT = c->iT();
  H.kL = c->L;
  H.kLK = c->L + c->K;
  H.alpha = c->alpha;
  H.dnum = c->dnum;
  H.kdnum = c->dnum;
  {
    // mod-up work items and the two-prime digit constants
    const uint32_t LK = c->L + c->K;
    H.mu_n[0] = H.mu_n[1] = 0;
    for (uint32_t g = 0; g < c->dnum; ++g)
      for (uint32_t j = 0; j < LK; ++j) {
        const bool own = j < c->L && j / c->alpha == g;
        for (int skip = 0; skip < 2; ++skip) {
          if (skip && own) continue;
          H.mu_g[skip][H.mu_n[skip]] = (uint8_t)g;
          H.mu_j[skip][H.mu_n[skip]] = (uint8_t)j;
          ++H.mu_n[skip];
        }
      }
    uint64_t qlo = ~0ull, qhi = 0;
    for (uint32_t j = 0; j < LK; ++j) {
      qlo = std::min(qlo, qp[j]);
      qhi = std::max(qhi, qp[j]);
    }
    H.modup_lazy_a = qhi / 6 < qlo ? 1u : 0u;
    for (uint32_t g = 0; g < c->dnum; ++g) {
      const uint32_t a = g * c->alpha;
      if (c->alpha < 2 || a + 1 >= c->L) continue;     // single-prime digit
      const uint64_t qa = qp[a], qb = qp[a + 1];
      if (qa / 2 >= qb) return fail(LOLA_E_PARAM, "a two-prime digit needs its first prime below twice its second");
      H.grp_inv[g] = invmod_h(qa % qb, qb);
      H.grp_inv_s[g] = shoup_h(H.grp_inv[g], qb);
      for (uint32_t j = 0; j < LK; ++j) {
        H.grp_qa[g][j] = qa % qp[j];
        H.grp_qa_s[g][j] = shoup_h(H.grp_qa[g][j], qp[j]);
      }
    }
  }
  const uint64_t n = c->n;
  std::vector<uint64_t> tw((size_t)4 * np * n);
  uint64_t* twf = tw.data();                  // [np][n][2]: (w, w')
  uint64_t* twi = twf + (size_t)2 * np * n;
  for (uint32_t pi = 0; pi < np; ++pi) {
    const uint64_t q = c->primes[pi];
    PrimeDev& P = H.pr[pi];
    P.q = q;
    uint64_t inv = 1;  // q^-1 mod 2^64 by Newton iteration
    for (int it = 0; it < 6; ++it) inv *= 2 - q * inv;
    P.qinv = (uint64_t)(0 - inv);
    const uint64_t r1 = (uint64_t)(((u128)1 << 64) % q);
    P.r2 = mulmod_h(r1, r1, q);
    P.f64 = (uint64_t)(~0ull / q);
    P.ninv = invmod_h(n % q, q);
    P.ninv_s = shoup_h(P.ninv, q);
    P.ninvr = mulmod_h(P.ninv, r1, q);
    P.ninvr_s = shoup_h(P.ninvr, q);
    const uint64_t psi = smallest_root_2n(q, c->n);
    const uint64_t ipsi = invmod_h(psi, q);
    std::vector<uint64_t> pw(n), ipw(n);   // psi^k, psi^-k
    pw[0] = ipw[0] = 1;
    for (uint32_t k2 = 1; k2 < n; ++k2) {
      pw[k2] = mulmod_h(pw[k2 - 1], psi, q);
      ipw[k2] = mulmod_h(ipw[k2 - 1], ipsi, q);
    }
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t e = brev_h(i, c->logn);
      const uint64_t w = pw[e], wi = ipw[e];
      twf[((size_t)pi * n + i) * 2] = w;
      twf[((size_t)pi * n + i) * 2 + 1] = shoup_h(w, q);
      twi[((size_t)pi * n + i) * 2] = wi;
      twi[((size_t)pi * n + i) * 2 + 1] = shoup_h(wi, q);
    }
  }
  // exact conversion constants
  std::vector<uint64_t> Qb(qp.begin(), qp.begin() + c->L);
  mrc_table(Qb, H.mrcQ);
  mrc_table(aux, H.mrcB);
  for (uint32_t j = 0; j < c->M; ++j) {
    const uint64_t b = aux[j];
    for (uint32_t k2 = 0; k2 < c->L; ++k2) {
      H.wQB[k2][j] = prefix_prod_mod(Qb, (int)k2, b);
      H.wQB_s[k2][j] = shoup_h(H.wQB[k2][j], b);
    }
    H.QmodB[j] = prefix_prod_mod(Qb, (int)c->L, b);
    H.QinvB[j] = invmod_h(H.QmodB[j], b);
    H.QinvB_s[j] = shoup_h(H.QinvB[j], b);
  }
  for (uint32_t i = 0; i < c->L; ++i) {
    const uint64_t q = Qb[i];
    for (uint32_t k2 = 0; k2 < c->M; ++k2) {
      H.wBQ[k2][i] = prefix_prod_mod(aux, (int)k2, q);
      H.wBQ_s[k2][i] = shoup_h(H.wBQ[k2][i], q);
    }
    H.BmodQ[i] = prefix_prod_mod(aux, (int)c->M, q);
  }
  for (uint32_t ti = 0; ti < c->kt; ++ti) {
    const uint64_t t = ts[ti];
    for (uint32_t i = 0; i < c->L; ++i) {
      H.tQ[ti][i] = t % Qb[i];
      H.tQ_s[ti][i] = shoup_h(H.tQ[ti][i], Qb[i]);
      // floor(Q / t) mod q_i = -(Q mod t) t^-1 mod q_i   (q_i divides Q)
      const uint64_t Qt = prefix_prod_mod(Qb, (int)c->L, t);
      const uint64_t d = mulmod_h((Qb[i] - Qt % Qb[i]) % Qb[i], invmod_h(t % Qb[i], Qb[i]), Qb[i]);
      H.deltaQ[ti][i] = d;
      H.deltaQ_s[ti][i] = shoup_h(d, Qb[i]);
    }
    for (uint32_t j = 0; j < c->M; ++j) {
      H.tB[ti][j] = t % aux[j];
      H.tB_s[ti][j] = shoup_h(H.tB[ti][j], aux[j]);
    }
    for (uint32_t k2 = 0; k2 < c->L; ++k2) {
      H.wQT[k2][ti] = prefix_prod_mod(Qb, (int)k2, t);
      H.wQT_s[k2][ti] = shoup_h(H.wQT[k2][ti], t);
    }
    H.QinvT[ti] = invmod_h(prefix_prod_mod(Qb, (int)c->L, t), t);
    H.QinvT_s[ti] = shoup_h(H.QinvT[ti], t);
  }
  // P = product of the special primes, reduced mod each ciphertext prime
  for (uint32_t i = 0; i < c->L; ++i) {
    const uint64_t q = Qb[i];
    uint64_t Pq = 1 % q;
    for (uint32_t k2 = 0; k2 < c->K; ++k2) Pq = mulmod_h(Pq, qp[c->L + k2] % q, q);
    H.PmodQ[i] = Pq;
    H.PmodQ_s[i] = shoup_h(H.PmodQ[i], q);
    H.PinvQ[i] = c->K ? invmod_h(Pq, q) : 1;
    H.PinvQ_s[i] = shoup_h(H.PinvQ[i], q);
    const uint64_t r1 = (uint64_t)(((u128)1 << 64) % q);
    H.PmontQ[i] = mulmod_h(Pq, r1, q);
    H.KskR2[i] = mulmod_h(H.pr[i].r2, H.PinvQ[i], q);
    H.KskOut[i] = H.PmodQ[i];
    if (c->K == 2) {
      H.P1PinvQ[i] = mulmod_h(qp[c->L] % q, H.PinvQ[i], q);
      H.P1PinvQ_s[i] = shoup_h(H.P1PinvQ[i], q);
    }
  }
  if (c->K == 2) {
    const uint64_t P1 = qp[c->L], P2 = qp[c->L + 1];
    H.P1invP2 = invmod_h(P1 % P2, P2);
    H.P1invP2_s = shoup_h(H.P1invP2, P2);
    const u128 half = ((u128)P1 * P2 - 1) / 2;
    H.ph1 = (uint64_t)(half % P1);
    H.phv = (uint64_t)(half / P1);
  }
  for (uint32_t i = c->L; i < c->L + c->K; ++i) {
    H.KskR2[i] = H.pr[i].r2;
    H.KskOut[i] = 1;
  }
  // slot map for the plaintext transform mod t: NTT position k holds the
  // value at psi^(2 brev(k) + 1); slot j sits at psi^(3^j), slot n/2 + j at psi^(-3^j)
  std::vector<uint32_t> slot_at_pos(n);
  {
    uint64_t e = 1;
    for (uint32_t j = 0; j < n / 2; ++j) {
      const uint32_t pos0 = brev_h((uint32_t)((e - 1) / 2), c->logn);
      const uint32_t pos1 = brev_h((uint32_t)((two_n - e - 1) / 2), c->logn);
      slot_at_pos[pos0] = j;
      slot_at_pos[pos1] = (uint32_t)(n / 2 + j);
      e = (e * 3) % two_n;
    }
  }
  int rc;
  if ((rc = c->d_tw.alloc(tw.size() * 8)) != LOLA_OK) return rc;
  LOLA_CUDA_TRY(cudaMemcpy(c->d_tw.p, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));
  H.tw_fwd = c->d_tw.u64();
  H.tw_inv = H.tw_fwd + (size_t)2 * np * n;
  if ((rc = c->d_slotpos.alloc(n * 4)) != LOLA_OK) return rc;
  LOLA_CUDA_TRY(cudaMemcpy(c->d_slotpos.p, slot_at_pos.data(), n * 4, cudaMemcpyHostToDevice));
  if ((rc = c->d_const.alloc(sizeof(CtxDev))) != LOLA_OK) return rc;
  LOLA_CUDA_TRY(cudaMemcpy(c->d_const.p, &H, sizeof(CtxDev), cudaMemcpyHostToDevice));
  c->dev = (CtxDev*)c->d_const.p;
  return LOLA_OK;
}

int ctx_create(const lola_params* p, int device, Ctx** out) {
  if (!p || !out) return fail(LOLA_E_PARAM, "null argument");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(LOLA_E_CUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return fail(LOLA_E_PARAM, "bad device index");
  LOLA_CUDA_TRY(cudaSetDevice(device));
  Ctx* c = new Ctx();
  c->device = device;
  int rc = build_ctx(c, p);
  if (rc != LOLA_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return LOLA_OK;
}

int ctx_level(Ctx* c, uint32_t Lv, Ctx** out) {
  Ctx* r = c->root;
  if (Lv == r->L) {
    *out = r;
    return LOLA_OK;
  }
  if (Lv < 1 || Lv > r->L) return fail(LOLA_E_PARAM, "level out of range");
  auto it = r->levels.find(Lv);
  if (it != r->levels.end()) {
    *out = it->second.get();
    return LOLA_OK;
  }
  std::vector<uint64_t> q(r->primes.begin(), r->primes.begin() + Lv);
  q.insert(q.end(), r->primes.begin() + r->L, r->primes.begin() + r->L + r->K);
  std::vector<uint64_t> t(r->primes.begin() + r->iT(), r->primes.begin() + r->iT() + r->kt);
  lola_params p{r->n, Lv, r->K, q.data(), r->kt, t.data(), r->alpha};
  std::unique_ptr<Ctx> lc(new Ctx());
  lc->device = r->device;
  LOLA_CUDA_TRY(cudaSetDevice(r->device));
  int rc = build_ctx(lc.get(), &p);
  if (rc != LOLA_OK) return rc;
  lc->root = r;
  lc->host.kL = r->L;
  lc->host.kLK = r->L + r->K;
  lc->host.kdnum = r->dnum;
  LOLA_CUDA_TRY(cudaMemcpy(lc->d_const.p, &lc->host, sizeof(CtxDev), cudaMemcpyHostToDevice));
  *out = lc.get();
  r->levels[Lv] = std::move(lc);
  return LOLA_OK;
}

void ctx_destroy(Ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  c->levels.clear();
  for (int k2 = 0; k2 < KI_COUNT; ++k2) prof_collect(c, k2);
  for (auto& pr : c->prof.pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  delete c;
}

int profile_enable(Ctx* c, int kind, int on) {
  if (!c || kind < -1 || kind >= KI_COUNT) return fail(LOLA_E_PARAM, "bad profile kind");
  for (int k2 = (kind < 0 ? 0 : kind); k2 < (kind < 0 ? KI_COUNT : kind + 1); ++k2) {
    prof_collect(c, k2);
    c->prof.on[k2] = on != 0;
    c->prof.ms[k2] = 0;
    c->prof.launches[k2] = 0;
    c->prof.units[k2] = 0;
  }
  return LOLA_OK;
}

int profile_read(Ctx* c, int kind, double* ms, uint64_t* launches, uint64_t* units) {
  if (!c || kind < 0 || kind >= KI_COUNT) return fail(LOLA_E_PARAM, "bad profile kind");
  prof_collect(c, kind);
  if (ms) *ms = c->prof.ms[kind];
  if (launches) *launches = c->prof.launches[kind];
  if (units) *units = c->prof.units[kind];
  return LOLA_OK;
}

}  // namespace lola
