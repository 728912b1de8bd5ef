// BFV operations (paper Sec. 3.1): key generation, encryption, decryption,
// rotation (Galois automorphism + key switching), ct x ct with exact
// scaling + relinearisation, plaintext encoding.  Host code that sequences
// the kernels; all arithmetic on ciphertexts runs on the device.
#include <string.h>

#include <algorithm>

#include "gauss_cdt.h"
#include "he.h"
#include "sampler.h"

namespace lola {

// ------------------------------------------------------------------ sampler
void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    const u128 p0 = (u128)0xD2E7470EE14C6C93ull * c0;
    const u128 p1 = (u128)0xCA5A826395121157ull * c2;
    const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c1 ^ k0;
    const uint64_t n1 = (uint64_t)p1;
    const uint64_t n2 = (uint64_t)(p0 >> 64) ^ c3 ^ k1;
    const uint64_t n3 = (uint64_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B97F4A7C15ull;   // key schedule: Weyl increments
    k1 += 0xBB67AE8584CAA73Bull;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint64_t PhiloxStream::next() {
  const uint64_t blk = word_ >> 2;
  if (blk != block_id_) {
    const uint64_t ctr[4] = {blk, tag_, a_, b_};
    const uint64_t key[2] = {seed_, 0};
    philox4x64_10(ctr, key, block_);
    block_id_ = blk;
  }
  return block_[word_++ & 3];
}

void sample_uniform(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t q, uint64_t* out, size_t n) {
  PhiloxStream st(seed, tag, a, b);
  int bits = 64 - __builtin_clzll(q);
  const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
  for (size_t i = 0; i < n;) {
    const uint64_t x = st.next() & mask;
    if (x < q) out[i++] = x;
  }
}

void sample_ternary(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, int64_t* out, size_t n) {
  PhiloxStream st(seed, tag, a, b);
  const uint64_t limit = 3 * (~0ull / 3);   // 3 floor(2^64/3) = 2^64 - 1 when computed this way
  for (size_t i = 0; i < n;) {
    const uint64_t w = st.next();
    if (w >= limit) continue;
    const uint64_t r = w % 3;
    out[i++] = r == 0 ? 0 : (r == 1 ? 1 : -1);
  }
}

void sample_gaussian(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, int64_t* out, size_t n) {
  PhiloxStream st(seed, tag, a, b);
  for (size_t i = 0; i < n; ++i) {
    const uint64_t w = st.next();
    const uint64_t u = w & 0x7FFFFFFFFFFFFFFFull;
    int64_t k = 0;
    while (u >= kGaussCdt[k]) ++k;
    out[i] = (w >> 63) ? -k : k;
  }
}

// ----------------------------------------------------------------- helpers
static PrimeMap prime_map(uint32_t limbs, uint32_t first = 0) {
  PrimeMap m{};
  for (uint32_t l = 0; l < limbs && l < 32; ++l) m.p[l] = (uint8_t)(first + l);
  return m;
}

// stream-ordered scratch
struct AsyncBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  int alloc(size_t bytes, cudaStream_t st) {
    s = st;
    if (!bytes) return LOLA_OK;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(LOLA_E_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    return LOLA_OK;
  }
  ~AsyncBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  template <class T>
  T* as() const { return (T*)p; }
};

#define TRY(x)                \
  do {                        \
    int _rc = (x);            \
    if (_rc != LOLA_OK) return _rc; \
  } while (0)

// --------------------------------------------------------------- key switching
// scratch: digits [count][L][n], mod-up limbs D [count][dnum][L+K][n], x_P
// [count][2][K][n]; the inner products live in place over D's digit rows 0
// and 1 (a separate [count][2][L+K][n] area when there is one digit).
// tau_g(c0) has no area: rotate() always has the inner product gather it
// from the input (c0_gather), and lola_rotate_noalloc's size check relies on
// this count.
size_t rotate_scratch_words(const Ctx* c, size_t count) {
  const size_t LK = c->L + c->K;
  size_t w = count * (c->L + c->dnum * LK + 2 * (size_t)c->K) * (size_t)c->n;   // digits, D, x_P
  if (c->dnum < 2) w += count * 2 * LK * (size_t)c->n;
  return w;
}

// Mod-up, inner product and (special prime) mod-down, shared by rotation
// (have_diag: decompose wrote the diagonal limbs D[i][i]) and
// relinearisation.
static int ks_switch(Ctx* c, KsDev& a, uint64_t* extra_acc, bool have_diag, cudaStream_t s) {
  const size_t n = c->n, LK = c->L + c->K;
  if (!c->K) {
    TRY(k::ks_modup(c, a, have_diag, s));
    return k::ks_ip(c, a, true, s);
  }
  if (c->dnum >= 2) {
    a.acc = a.D;
    a.acc_stride = c->dnum * LK * n;
  } else {
    a.acc = extra_acc;
    a.acc_stride = 2 * LK * n;
  }
  TRY(k::ks_modup(c, a, have_diag, s));
  TRY(k::ks_ip(c, a, false, s));
  TRY(k::ks_intt_p(c, a, s));
  return k::ks_moddown(c, a, s);
}

int rotate(Ctx* c, const uint64_t* in, uint64_t* out, const uint64_t* accum, size_t count, const RotSpec& r,
           uint64_t* scratch, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  KsDev a{};
  a.c0 = in;
  a.c1 = in;
  a.add1 = nullptr;
  a.accum = accum;
  a.out = out;
  a.dig = scratch;
  a.D = a.dig + count * L * n;
  a.xP = a.D + count * c->dnum * LK * n;
  a.c0_gather = 1;                            // the inner product gathers tau_g(c0)
  a.count = count;
  a.d_gal = r.d_gal;
  a.gal = r.gal;
  a.d_keys = r.d_keys;
  a.key = r.key;
  a.gal_div = r.div ? r.div : 1;
  TRY(k::ks_decompose(c, a, s));
  return ks_switch(c, a, a.xP + count * 2 * c->K * n, true, s);
}

// Hoisted rotations: every one of `count` ciphertexts rotated by each of
// S steps, out = [S][count] ciphertexts.  The digits of c1 are decomposed
// and raised to Q * P once (decompose with the identity, mod-up); each
// step then gathers tau_g(D) and tau_g(c0) inside the inner product and
// runs INTT mod P and mod-down for all S * count outputs in one launch each.
// steps per inner-product launch: at most ~1024 outputs, at least one step
static size_t hoisted_chunk(size_t count, size_t S) { return std::min(S, std::max<size_t>(1, 1024 / count)); }

size_t rotate_hoisted_scratch_words(const Ctx* c, size_t count, size_t S) {
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  return count * (L + c->dnum * LK) * n + hoisted_chunk(count, S) * count * (2 * LK + 2 * c->K) * n;
}

int rotate_hoisted(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, size_t S, const uint32_t* d_gal,
                   const uint64_t* const* d_keys, uint64_t* scratch, cudaStream_t s) {
  if (!count || !S) return LOLA_OK;
  const size_t chunk = hoisted_chunk(count, S);
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  KsDev a{};
  a.c0 = in;
  a.c1 = in;
  a.dig = scratch;
  a.D = a.dig + count * L * n;
  a.count = count;
  a.gal = 1;
  a.gal_div = 1;
  TRY(k::ks_decompose(c, a, s));
  TRY(k::ks_modup(c, a, true, s));
  for (size_t s0 = 0; s0 < S; s0 += chunk) {
    const size_t sc = std::min(chunk, S - s0);
    KsDev b{};
    b.c0 = in;
    b.out = out + s0 * count * c->ct_words();
    b.D = a.D;
    b.acc = a.D + count * c->dnum * LK * n;
    b.acc_stride = 2 * LK * n;
    b.xP = b.acc + sc * count * 2 * LK * n;
    b.count = sc * count;
    b.d_gal = d_gal + s0;
    b.d_keys = d_keys + s0;
    b.gal_div = (uint32_t)count;
    b.src_mod = (uint32_t)count;
    b.ip_gather = 1;
    if (!c->K) {
      TRY(k::ks_ip(c, b, true, s));
      continue;
    }
    TRY(k::ks_ip(c, b, false, s));
    TRY(k::ks_intt_p(c, b, s));
    TRY(k::ks_moddown(c, b, s));
  }
  return LOLA_OK;
}

// Rotate-sum (several rotate-and-sum doubling steps in one key switch): c1
// is decomposed without an automorphism and raised to Q * P once; one inner
// product adds, for every element g, the gathered digits tau_g(D) times g's
// key, plus x and every tau_g(c0); one INTT mod P and one mod-down follow.
// scratch: digits [count][L][n], D [count][dnum][L+K][n], the inner
// products [count][2][L+K][n] (not over D: the gathers read all of it), x_P
// [count][2][K][n].
size_t rotate_sum_scratch_words(const Ctx* c, size_t count) {
  const size_t LK = c->L + c->K;
  return count * (c->L + c->dnum * LK + 2 * LK + 2 * (size_t)c->K) * (size_t)c->n;
}

int rotate_sum(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, uint32_t G, const uint32_t* d_gal,
               const uint64_t* const* d_keys, uint32_t gal_div, uint64_t* scratch, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  if (!G) {
    LOLA_CUDA_TRY(cudaMemcpyAsync(out, in, count * c->ct_words() * 8, cudaMemcpyDeviceToDevice, s));
    return LOLA_OK;
  }
  KsDev a{};
  a.c0 = in;
  a.c1 = in;
  a.accum = in;
  a.out = out;
  a.dig = scratch;
  a.D = a.dig + count * L * n;
  a.acc = a.D + count * c->dnum * LK * n;
  a.acc_stride = 2 * LK * n;
  a.xP = a.acc + count * 2 * LK * n;
  a.count = count;
  a.gal = 1;                                  // decompose: no automorphism
  a.gal_div = 1;
  TRY(k::ks_decompose(c, a, s));
  TRY(k::ks_modup(c, a, true, s));
  a.d_gal = d_gal;
  a.d_keys = d_keys;
  a.gal_div = gal_div ? gal_div : 1;
  a.gsum = G;
  TRY(k::ks_ip_sum(c, a, c->K == 0, s));
  if (!c->K) return LOLA_OK;
  TRY(k::ks_intt_p(c, a, s));
  return k::ks_moddown(c, a, s);
}

// ------------------------------------------------------- modulus switching
// scratch: the dropped limbs in coefficient form [count][2][n], and two
// intermediate ciphertext arrays when more than one prime is dropped
size_t mod_switch_scratch_words(const Ctx* c, size_t count, uint32_t L_from, uint32_t L_to) {
  if (L_from <= L_to) return 0;
  size_t w = count * 2 * (size_t)c->n;
  if (L_from - L_to > 1) w += 2 * count * 2 * (size_t)(L_from - 1) * c->n;
  return w;
}

int mod_switch(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, uint32_t L_from, uint32_t L_to,
               uint64_t* scratch, cudaStream_t s) {
  c = c->root;
  if (L_to < 1 || L_to > L_from || L_from > c->L) return fail(LOLA_E_PARAM, "mod switch: bad levels");
  if (!count) return LOLA_OK;
  const size_t n = c->n;
  if (L_from == L_to) {
    if (in != out) LOLA_CUDA_TRY(cudaMemcpyAsync(out, in, count * 2 * L_from * n * 8, cudaMemcpyDeviceToDevice, s));
    return LOLA_OK;
  }
  uint64_t* top = scratch;
  uint64_t* tmp[2] = {top + count * 2 * n, top + count * 2 * n + count * 2 * (L_from - 1) * n};
  const uint64_t* src = in;
  for (uint32_t L1 = L_from; L1 > L_to; --L1) {
    uint64_t* dst = (L1 - 1 == L_to) ? out : tmp[(L_from - L1) & 1];
    TRY(k::mod_switch_drop(c, src, top, dst, count, L1, s));
    src = dst;
  }
  return LOLA_OK;
}

// ---------------------------------------------------------- ct x ct (Sec. 3.1 (x))
size_t multiply_scratch_words(const Ctx* c, size_t count, bool square) {
  const size_t n = c->n, L = c->L, M = c->M, LK = c->L + c->K;
  size_t w = count * 2 * L * n + count * 2 * M * n;   // X, XB
  if (!square) w *= 2;                                 // Y, YB
  w += count * 3 * (L + M) * n;                        // T
  w += count * 2 * L * n + count * L * n;              // E, DIG
  w += count * c->dnum * LK * n + count * 2 * c->K * n;   // D, xP
  if (c->dnum < 2) w += count * 2 * LK * n;            // inner products (one digit)
  return w;
}

int multiply(Ctx* c, const uint64_t* x, const uint64_t* y, uint64_t* out, size_t count, const uint32_t* d_tidx,
             uint32_t tidx_div, const uint64_t* relin_key, uint64_t* scratch, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const bool square = (x == y);
  const size_t n = c->n, L = c->L, M = c->M, LK = c->L + c->K;
  uint64_t* X = scratch;
  uint64_t* XB = X + count * 2 * L * n;
  uint64_t* Y = X;
  uint64_t* YB = XB;
  uint64_t* next = XB + count * 2 * M * n;
  if (!square) {
    Y = next;
    YB = Y + count * 2 * L * n;
    next = YB + count * 2 * M * n;
  }
  uint64_t* T = next;
  uint64_t* E = T + count * 3 * (L + M) * n;
  uint64_t* DIG = E + count * 2 * L * n;
  uint64_t* D = DIG + count * L * n;
  uint64_t* xP = D + count * c->dnum * LK * n;

  PrimeMap qmap = prime_map(L), bmap = prime_map(M, c->iB());
  PrimeMap qbmap{};
  for (uint32_t l = 0; l < L + M; ++l) qbmap.p[l] = (uint8_t)(l < L ? l : c->iB() + (l - L));
  // centered lift of x (and y) to the auxiliary basis, in NTT form there
  TRY(k::ntt_inv_map(c, x, X, count * 2 * L, L, qmap, false, s));
  TRY(k::lift_q_to_b(c, X, XB, count * 2, s));
  TRY(k::ntt_fwd_map(c, XB, XB, count * 2 * M, M, bmap, s));
  if (!square) {
    TRY(k::ntt_inv_map(c, y, Y, count * 2 * L, L, qmap, false, s));
    TRY(k::lift_q_to_b(c, Y, YB, count * 2, s));
    TRY(k::ntt_fwd_map(c, YB, YB, count * 2 * M, M, bmap, s));
  }
  // tensor over Q u B, back to coefficients, exact t/Q rounding
  TRY(k::tensor(c, x, XB, y, YB, T, count, s));
  TRY(k::ntt_inv_map(c, T, T, count * 3 * (L + M), L + M, qbmap, true, s));
  TRY(k::scale_round(c, T, d_tidx, tidx_div, E, DIG, count, s));
  TRY(k::ntt_fwd_map(c, E, E, count * 2 * L, L, qmap, s));
  // relinearisation: key-switch part 2 (digits already in coefficient form)
  KsDev a{};
  a.c0 = E;
  a.add1 = E;
  a.out = out;
  a.dig = DIG;
  a.D = D;
  a.xP = xP;
  a.count = count;
  a.gal = 1;
  a.key = relin_key;
  a.gal_div = 1;
  return ks_switch(c, a, xP + count * 2 * c->K * n, false, s);
}

// --------------------------------------------------------------------- keys
static int gen_switch_key(Ctx* c, const DevBuf& s_mont, const uint64_t* d_sfrom, uint64_t key_id, uint64_t seed,
                          std::shared_ptr<SwitchKey>* out, cudaStream_t s) {
  const size_t n = c->n, D = c->dnum, LK = c->L + c->K;
  std::vector<int64_t> e(D * n);
  std::vector<uint64_t> a(D * LK * n);
  for (size_t g = 0; g < D; ++g) {          // one row per digit (group of alpha primes)
    sample_gaussian(seed, TAG_KSK_E, key_id, g, e.data() + g * n, n);
    for (size_t j = 0; j < LK; ++j)
      sample_uniform(seed, TAG_KSK_A, key_id, g * 256 + j, c->primes[j], a.data() + (g * LK + j) * n, n);
  }
  AsyncBuf de, da, dE;
  TRY(de.alloc(e.size() * 8, s));
  TRY(da.alloc(a.size() * 8, s));
  TRY(dE.alloc(a.size() * 8, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(de.p, e.data(), e.size() * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(da.p, a.data(), a.size() * 8, cudaMemcpyHostToDevice, s));
  PrimeMap lk = prime_map(LK);
  TRY(k::ntt_fwd_map(c, da.as<uint64_t>(), da.as<uint64_t>(), D * LK, LK, lk, s));
  TRY(k::ntt_fwd_from_signed(c, de.as<int64_t>(), dE.as<uint64_t>(), D, LK, 0, s));
  auto key = std::make_shared<SwitchKey>();
  TRY(key->buf.alloc(2 * D * LK * n * 8));
  TRY(k::keygen_switch(c, da.as<uint64_t>(), dE.as<uint64_t>(), s_mont.u64(), d_sfrom, key->buf.u64(), s));
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  *out = key;
  return LOLA_OK;
}

int keygen(Ctx* c, uint64_t seed, const int32_t* steps, size_t n_steps, uint32_t flags, KeySet** secret,
           KeySet** eval) {
  if (!secret) return fail(LOLA_E_PARAM, "null output");
  *secret = nullptr;
  if (eval) *eval = nullptr;
  for (size_t i = 0; i < n_steps; ++i)
    if (steps[i] <= 0 || (uint32_t)steps[i] >= c->n / 2) return fail(LOLA_E_PARAM, "rotation step out of range");
  LOLA_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = nullptr;
  LOLA_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  } guard{s};
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  std::unique_ptr<KeySet> ks(new KeySet());
  ks->ctx = c;
  ks->ev = std::make_shared<EvalKeys>();
  // secret: ternary
  ks->s_coeff.resize(n);
  sample_ternary(seed, TAG_SECRET, 0, 0, ks->s_coeff.data(), n);
  AsyncBuf ds;
  TRY(ds.alloc(n * 8, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(ds.p, ks->s_coeff.data(), n * 8, cudaMemcpyHostToDevice, s));
  TRY(ks->s_ntt.alloc(LK * n * 8));
  TRY(ks->s_mont.alloc(LK * n * 8));
  TRY(k::ntt_fwd_from_signed(c, ds.as<int64_t>(), ks->s_ntt.u64(), 1, LK, 0, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(ks->s_mont.p, ks->s_ntt.p, LK * n * 8, cudaMemcpyDeviceToDevice, s));
  PrimeMap lk = prime_map(LK);
  TRY(k::to_mont_map(c, ks->s_mont.u64(), LK, LK, lk, s));
  // public key over Q
  {
    std::vector<uint64_t> a(L * n);
    std::vector<int64_t> e(n);
    for (size_t j = 0; j < L; ++j) sample_uniform(seed, TAG_PK_A, j, 0, c->primes[j], a.data() + j * n, n);
    sample_gaussian(seed, TAG_PK_E, 0, 0, e.data(), n);
    AsyncBuf da, de, dE;
    TRY(da.alloc(L * n * 8, s));
    TRY(de.alloc(n * 8, s));
    TRY(dE.alloc(L * n * 8, s));
    LOLA_CUDA_TRY(cudaMemcpyAsync(da.p, a.data(), L * n * 8, cudaMemcpyHostToDevice, s));
    LOLA_CUDA_TRY(cudaMemcpyAsync(de.p, e.data(), n * 8, cudaMemcpyHostToDevice, s));
    PrimeMap qm = prime_map(L);
    TRY(k::ntt_fwd_map(c, da.as<uint64_t>(), da.as<uint64_t>(), L, L, qm, s));
    TRY(k::ntt_fwd_from_signed(c, de.as<int64_t>(), dE.as<uint64_t>(), 1, L, 0, s));
    TRY(ks->pk.alloc(2 * L * n * 8));
    TRY(k::neg_axpe(c, da.as<uint64_t>(), ks->s_mont.u64(), dE.as<uint64_t>(), ks->pk.u64(), L, s));
    LOLA_CUDA_TRY(cudaMemcpyAsync(ks->pk.u64() + L * n, da.p, L * n * 8, cudaMemcpyDeviceToDevice, s));
    TRY(k::to_mont_map(c, ks->pk.u64(), 2 * L, L, qm, s));
    LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  }
  ks->has_secret = ks->has_public = true;
  // relinearisation key: s' = s^2
  if (flags & LOLA_KEY_RELIN) {
    AsyncBuf s2;
    TRY(s2.alloc(LK * n * 8, s));
    TRY(k::axpy_mont_map(c, nullptr, ks->s_ntt.u64(), ks->s_mont.u64(), s2.as<uint64_t>(), LK, LK, lk, s));
    TRY(gen_switch_key(c, ks->s_mont, s2.as<uint64_t>(), 0, seed, &ks->ev->relin, s));
  }
  // Galois keys: s' = tau_g(s)
  std::vector<uint32_t> gals;
  for (size_t i = 0; i < n_steps; ++i) gals.push_back(galois_for_step(c->n, steps[i]));
  if (flags & LOLA_KEY_ROW_SWAP) gals.push_back(galois_for_step(c->n, 0));
  for (uint32_t g : gals) {
    if (ks->ev->galois.count(g)) continue;
    AsyncBuf sg;
    TRY(sg.alloc(LK * n * 8, s));
    TRY(k::gal_permute(c, ks->s_ntt.u64(), sg.as<uint64_t>(), LK, g, s));
    std::shared_ptr<SwitchKey> key;
    TRY(gen_switch_key(c, ks->s_mont, sg.as<uint64_t>(), g, seed, &key, s));
    ks->ev->galois[g] = key;
  }
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  if (eval) {
    KeySet* e = new KeySet();
    e->ctx = c;
    e->ev = ks->ev;
    *eval = e;
  }
  *secret = ks.release();
  return LOLA_OK;
}

int keys_export(Ctx* c, const KeySet* ks, int what, int32_t step, uint64_t* host, size_t* words) {
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  size_t need = 0;
  const uint64_t* src = nullptr;
  uint32_t limbs = 0;
  switch (what) {
    case 0:
      if (!ks->has_secret) return fail(LOLA_E_STATE, "no secret key in this handle");
      need = n;
      break;
    case 1:
      if (!ks->has_public) return fail(LOLA_E_STATE, "no public key in this handle");
      need = 2 * L * n;
      src = ks->pk.u64();
      limbs = L;
      break;
    case 2:
      if (!ks->ev->relin) return fail(LOLA_E_NOKEY, "no relinearisation key");
      need = 2 * c->dnum * LK * n;
      src = ks->ev->relin->buf.u64();
      limbs = LK;
      break;
    case 3: {
      if (step < 0 || (uint32_t)step >= c->n / 2) return fail(LOLA_E_PARAM, "bad step");
      const SwitchKey* k2 = ks->galois_key(galois_for_step(c->n, step));
      if (!k2) return fail(LOLA_E_NOKEY, "no Galois key for this step");
      need = 2 * c->dnum * LK * n;
      src = k2->buf.u64();
      limbs = LK;
      break;
    }
    default:
      return fail(LOLA_E_PARAM, "bad key selector");
  }
  if (words) *words = need;
  if (!host) return LOLA_OK;
  if (what == 0) {
    for (size_t i = 0; i < n; ++i) host[i] = (uint64_t)ks->s_coeff[i];
    return LOLA_OK;
  }
  cudaStream_t s = nullptr;
  DevBuf tmp;
  TRY(tmp.alloc(need * 8));
  LOLA_CUDA_TRY(cudaMemcpy(tmp.p, src, need * 8, cudaMemcpyDeviceToDevice));
  PrimeMap pm = prime_map(limbs);
  TRY(k::to_mont_map(c, tmp.u64(), need / n, limbs, pm, s, what == 1 ? k::MONT_FROM : k::MONT_FROM_KSK));
  TRY(k::ntt_inv_map(c, tmp.u64(), tmp.u64(), need / n, limbs, pm, false, s));
  LOLA_CUDA_TRY(cudaMemcpy(host, tmp.p, need * 8, cudaMemcpyDeviceToHost));
  return LOLA_OK;
}

// -------------------------------------------------------------- encryption
int encode_plaintexts(Ctx* c, const int64_t* slots, const uint32_t* tidx, size_t count, uint64_t* d_out,
                      cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t n = c->n, L = c->L;
  std::vector<uint64_t> red(count * n);
  for (size_t i = 0; i < count; ++i) {
    const int64_t t = (int64_t)c->primes[c->iT() + tidx[i]];
    for (size_t j = 0; j < n; ++j) {
      int64_t v = slots[i * n + j] % t;
      red[i * n + j] = (uint64_t)(v < 0 ? v + t : v);
    }
  }
  AsyncBuf dsl, dco, dti;
  TRY(dsl.alloc(count * n * 8, s));
  TRY(dco.alloc(count * n * 8, s));
  TRY(dti.alloc(count * 4, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dsl.p, red.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dti.p, tidx, count * 4, cudaMemcpyHostToDevice, s));
  TRY(k::slots_to_coeff(c, dsl.as<uint64_t>(), dti.as<uint32_t>(), dco.as<uint64_t>(), count, s));
  TRY(k::encode_lift(c, dco.as<uint64_t>(), dti.as<uint32_t>(), d_out, count, L, true, s));
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  return LOLA_OK;
}

int encrypt(Ctx* c, const KeySet* ks, const int64_t* slots, size_t n_msg, uint64_t seed, uint64_t* d_out,
            cudaStream_t s) {
  if (!ks->has_public) return fail(LOLA_E_STATE, "no public key in this handle");
  const size_t n = c->n, L = c->L, kt = c->kt;
  const size_t count = n_msg * kt;
  if (!count) return LOLA_OK;
  std::vector<uint64_t> red(count * n);
  std::vector<uint32_t> tidx(count);
  std::vector<int64_t> u(count * n), e1(count * n), e2(count * n);
  for (size_t m = 0; m < n_msg; ++m)
    for (size_t ti = 0; ti < kt; ++ti) {
      const size_t id = m * kt + ti;
      const int64_t t = (int64_t)c->primes[c->iT() + ti];
      tidx[id] = (uint32_t)ti;
      for (size_t j = 0; j < n; ++j) {
        int64_t v = slots[m * n + j] % t;
        red[id * n + j] = (uint64_t)(v < 0 ? v + t : v);
      }
      sample_ternary(seed, TAG_ENC_U, id, 0, u.data() + id * n, n);
      sample_gaussian(seed, TAG_ENC_E1, id, 0, e1.data() + id * n, n);
      sample_gaussian(seed, TAG_ENC_E2, id, 0, e2.data() + id * n, n);
    }
  AsyncBuf dsl, dco, dti, du, de1, de2, dU, dM, dE2;
  TRY(dsl.alloc(count * n * 8, s));
  TRY(dco.alloc(count * n * 8, s));
  TRY(dti.alloc(count * 4, s));
  TRY(du.alloc(count * n * 8, s));
  TRY(de1.alloc(count * n * 8, s));
  TRY(de2.alloc(count * n * 8, s));
  TRY(dU.alloc(count * L * n * 8, s));
  TRY(dM.alloc(count * L * n * 8, s));
  TRY(dE2.alloc(count * L * n * 8, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dsl.p, red.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dti.p, tidx.data(), count * 4, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(du.p, u.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(de1.p, e1.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(de2.p, e2.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  TRY(k::slots_to_coeff(c, dsl.as<uint64_t>(), dti.as<uint32_t>(), dco.as<uint64_t>(), count, s));
  TRY(k::ntt_fwd_from_signed(c, du.as<int64_t>(), dU.as<uint64_t>(), count, L, 0, s));
  TRY(k::enc_msg(c, dco.as<uint64_t>(), de1.as<int64_t>(), dti.as<uint32_t>(), dM.as<uint64_t>(), count, s));
  TRY(k::ntt_fwd_from_signed(c, de2.as<int64_t>(), dE2.as<uint64_t>(), count, L, 0, s));
  TRY(k::enc_combine(c, dM.as<uint64_t>(), dE2.as<uint64_t>(), dU.as<uint64_t>(), ks->pk.u64(), d_out, count, s));
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  return LOLA_OK;
}

int decrypt_residues(Ctx* c, const KeySet* ks, const uint64_t* d_ct, size_t n_msg, uint64_t* host_slots,
                     cudaStream_t s) {
  if (!ks->has_secret) return fail(LOLA_E_STATE, "no secret key in this handle");
  const size_t n = c->n, L = c->L, kt = c->kt;
  const size_t count = n_msg * kt;
  if (!count) return LOLA_OK;
  std::vector<uint32_t> tidx(count);
  for (size_t i = 0; i < count; ++i) tidx[i] = (uint32_t)(i % kt);
  AsyncBuf dX, dti, dm, dsl;
  TRY(dX.alloc(count * L * n * 8, s));
  TRY(dti.alloc(count * 4, s));
  TRY(dm.alloc(count * n * 8, s));
  TRY(dsl.alloc(count * n * 8, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dti.p, tidx.data(), count * 4, cudaMemcpyHostToDevice, s));
  TRY(k::dec_phase(c, d_ct, ks->s_mont.u64(), dX.as<uint64_t>(), count, s));
  PrimeMap qm = prime_map(L);
  TRY(k::ntt_inv_map(c, dX.as<uint64_t>(), dX.as<uint64_t>(), count * L, L, qm, false, s));
  TRY(k::decrypt_round(c, dX.as<uint64_t>(), dti.as<uint32_t>(), dm.as<uint64_t>(), count, s));
  TRY(k::coeff_to_slots(c, dm.as<uint64_t>(), dti.as<uint32_t>(), dsl.as<uint64_t>(), count, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(host_slots, dsl.p, count * n * 8, cudaMemcpyDeviceToHost, s));
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  return LOLA_OK;
}

int to_coeff(Ctx* c, const uint64_t* d_ct, uint64_t* d_out, size_t count, cudaStream_t s) {
  PrimeMap qm = prime_map(c->L);
  return k::ntt_inv_map(c, d_ct, d_out, count * 2 * c->L, c->L, qm, false, s);
}

int from_coeff(Ctx* c, const uint64_t* d_in, uint64_t* d_out, size_t count, cudaStream_t s) {
  PrimeMap qm = prime_map(c->L);
  return k::ntt_fwd_map(c, d_in, d_out, count * 2 * c->L, c->L, qm, s);
}

}  // namespace lola
