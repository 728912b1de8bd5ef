// C-ABI entry points (include/lola.h).  Argument checking and marshalling
// only; the work happens in he.cu / net.cu and the kernels.
#include <string.h>

#include <algorithm>
#include <new>

#include "net.h"

using namespace lola;

struct lola_ctx {
  Ctx* c;
};
struct lola_keys {
  KeySet* k;
};
struct lola_ct {
  Ct ct;
};
struct lola_net {
  Net* net;
  lola_ctx* ctx;
};

#define CHECK(cond, code, msg) \
  do {                         \
    if (!(cond)) return fail(code, msg); \
  } while (0)

#define TRY(x)                      \
  do {                              \
    int _rc = (x);                  \
    if (_rc != LOLA_OK) return _rc; \
  } while (0)

static cudaStream_t to_stream(void* s) { return (cudaStream_t)s; }

extern "C" {

const char* lola_last_error(void) { return lola::last_error(); }
const char* lola_version(void) { return "lola-gb300 0.1 (sm_103a)"; }

int lola_ctx_create(const lola_params* params, int device, lola_ctx** out) {
  CHECK(out, LOLA_E_PARAM, "null output");
  *out = nullptr;
  Ctx* c = nullptr;
  TRY(ctx_create(params, device, &c));
  *out = new lola_ctx{c};
  return LOLA_OK;
}

void lola_ctx_destroy(lola_ctx* ctx) {
  if (!ctx) return;
  ctx_destroy(ctx->c);
  delete ctx;
}

int lola_ctx_aux_primes(const lola_ctx* ctx, uint64_t* primes_out, uint32_t* count_out) {
  CHECK(ctx, LOLA_E_PARAM, "null context");
  const Ctx* c = ctx->c;
  if (count_out) *count_out = c->M;
  if (primes_out)
    for (uint32_t i = 0; i < c->M; ++i) primes_out[i] = c->primes[c->iB() + i];
  return LOLA_OK;
}

int lola_keygen(lola_ctx* ctx, uint64_t seed, const int32_t* rot_steps, size_t n_steps, uint32_t flags,
                lola_keys** secret_out, lola_keys** eval_out) {
  CHECK(ctx && secret_out, LOLA_E_PARAM, "null argument");
  CHECK(n_steps == 0 || rot_steps, LOLA_E_PARAM, "null step list");
  KeySet *s = nullptr, *e = nullptr;
  TRY(keygen(ctx->c, seed, rot_steps, n_steps, flags, &s, eval_out ? &e : nullptr));
  *secret_out = new lola_keys{s};
  if (eval_out) *eval_out = new lola_keys{e};
  return LOLA_OK;
}

void lola_keys_destroy(lola_keys* keys) {
  if (!keys) return;
  delete keys->k;
  delete keys;
}

int lola_keys_export(lola_ctx* ctx, const lola_keys* keys, int what, int32_t step, uint64_t* host,
                     size_t* words_out) {
  CHECK(ctx && keys, LOLA_E_PARAM, "null argument");
  return keys_export(ctx->c, keys->k, what, step, host, words_out);
}

static int new_ct(Ctx* c, size_t n_msg, lola_ct** out) {
  lola_ct* h = new (std::nothrow) lola_ct();
  CHECK(h, LOLA_E_NOMEM, "host allocation");
  h->ct.ctx = c;
  h->ct.n_msg = n_msg;
  int rc = h->ct.buf.alloc(h->ct.words() * 8);
  if (rc != LOLA_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return LOLA_OK;
}

int lola_ct_create(lola_ctx* ctx, size_t n_msg, lola_ct** out) {
  CHECK(ctx && out, LOLA_E_PARAM, "null argument");
  TRY(new_ct(ctx->c, n_msg, out));
  if ((*out)->ct.buf.bytes) LOLA_CUDA_TRY(cudaMemset((*out)->ct.buf.p, 0, (*out)->ct.buf.bytes));
  return LOLA_OK;
}

size_t lola_ct_messages(const lola_ct* ct) { return ct ? ct->ct.n_msg : 0; }
size_t lola_ct_bytes(const lola_ct* ct) { return ct ? ct->ct.buf.bytes : 0; }
uint64_t* lola_ct_data(lola_ct* ct) { return ct ? ct->ct.buf.u64() : nullptr; }

void lola_ct_destroy(lola_ct* ct) { delete ct; }

int lola_encrypt(lola_ctx* ctx, const lola_keys* keys, const int64_t* slots, size_t n_msg, uint64_t seed,
                 lola_ct** out) {
  CHECK(ctx && keys && out && (slots || !n_msg), LOLA_E_PARAM, "null argument");
  lola_ct* h = nullptr;
  TRY(new_ct(ctx->c, n_msg, &h));
  int rc = encrypt(ctx->c, keys->k, slots, n_msg, seed, h->ct.buf.u64(), nullptr);
  if (rc != LOLA_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return LOLA_OK;
}

int lola_encrypt_symmetric(lola_ctx* ctx, const lola_keys* keys, const int64_t* slots, size_t n_msg, uint64_t seed,
                           lola_ct** out) {
  CHECK(ctx && keys && out && (slots || !n_msg), LOLA_E_PARAM, "null argument");
  lola_ct* h = nullptr;
  TRY(new_ct(ctx->c, n_msg, &h));
  int rc = encrypt_symmetric(ctx->c, keys->k, slots, n_msg, seed, h->ct.buf.u64(), nullptr);
  if (rc != LOLA_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return LOLA_OK;
}

int lola_ct_upload_seeded(lola_ctx* ctx, lola_ct* ct, const uint64_t* host_c0, uint64_t seed, void* stream) {
  CHECK(ctx && ct && host_c0, LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  CHECK(ct->ct.L() == c->L, LOLA_E_PARAM, "seeded upload needs a ciphertext at the full level");
  const size_t count = ct->ct.n_msg * c->kt, limbs = (size_t)c->L * c->n;
  if (!count) return LOLA_OK;
  cudaStream_t s = to_stream(stream);
  LOLA_CUDA_TRY(cudaMemcpy2DAsync(ct->ct.buf.p, 2 * limbs * 8, host_c0, limbs * 8, limbs * 8, count,
                                  cudaMemcpyHostToDevice, s));
  return seeded_c1(c, ct->ct.buf.u64(), count, seed, 0, s);
}

// the context of a handle's level
static int ct_ctx(lola_ctx* ctx, const lola_ct* ct, Ctx** lc) { return ctx_level(ctx->c, ct->ct.L(), lc); }

int lola_decrypt_residues(lola_ctx* ctx, const lola_keys* keys, const lola_ct* ct, uint64_t* out) {
  CHECK(ctx && keys && ct && out, LOLA_E_PARAM, "null argument");
  Ctx* lc = nullptr;
  TRY(ct_ctx(ctx, ct, &lc));
  return decrypt_residues(lc, keys->k, ct->ct.buf.u64(), ct->ct.n_msg, out, nullptr);
}

int lola_decrypt_residues_level(lola_ctx* ctx, const lola_keys* keys, const uint64_t* d_ct, size_t n_msg,
                                uint32_t level, uint64_t* out) {
  CHECK(ctx && keys && (d_ct || !n_msg) && out, LOLA_E_PARAM, "null argument");
  Ctx* lc = nullptr;
  TRY(ctx_level(ctx->c, level, &lc));
  return decrypt_residues(lc, keys->k, d_ct, n_msg, out, nullptr);
}

uint32_t lola_ct_level(const lola_ct* ct) { return ct ? ct->ct.L() : 0; }

int lola_decrypt(lola_ctx* ctx, const lola_keys* keys, const lola_ct* ct, int64_t* out) {
  CHECK(ctx && keys && ct && out, LOLA_E_PARAM, "null argument");
  Ctx* c = nullptr;
  TRY(ct_ctx(ctx, ct, &c));
  const size_t n = c->n, kt = c->kt, m = ct->ct.n_msg;
  std::vector<uint64_t> res(m * kt * n);
  TRY(decrypt_residues(c, keys->k, ct->ct.buf.u64(), m, res.data(), nullptr));
  // Garner over t_0..t_{k-1}, then centered in (-T/2, T/2]  (Sec. 4.4)
  std::vector<uint64_t> t(kt);
  for (size_t i = 0; i < kt; ++i) t[i] = c->primes[c->iT() + i];
  typedef __int128 i128;
  u128 T = 1;
  for (size_t i = 0; i < kt; ++i) T *= t[i];
  for (size_t msg = 0; msg < m; ++msg)
    for (size_t j = 0; j < n; ++j) {
      u128 x = 0, prod = 1;
      for (size_t i = 0; i < kt; ++i) {
        const uint64_t r = res[(msg * kt + i) * n + j];
        // digit = (r - x) * prod^-1 mod t_i
        const uint64_t xm = (uint64_t)(x % t[i]), pm = (uint64_t)(prod % t[i]);
        const uint64_t dig = mulmod_h((r + t[i] - xm) % t[i], invmod_h(pm, t[i]), t[i]);
        x += prod * dig;
        prod *= t[i];
      }
      i128 v = (i128)x;
      if (x > T / 2) v = (i128)x - (i128)T;
      out[(msg * n + j) * 2] = (int64_t)(uint64_t)((u128)v);
      out[(msg * n + j) * 2 + 1] = (int64_t)(uint64_t)((u128)v >> 64);
    }
  return LOLA_OK;
}

int lola_ct_export(lola_ctx* ctx, const lola_ct* ct, uint64_t* host) {
  CHECK(ctx && ct && host, LOLA_E_PARAM, "null argument");
  Ctx* c = nullptr;
  TRY(ct_ctx(ctx, ct, &c));
  const size_t count = ct->ct.n_msg * c->kt;
  DevBuf tmp;
  TRY(tmp.alloc(count * c->ct_words() * 8));
  TRY(to_coeff(c, ct->ct.buf.u64(), tmp.u64(), count, nullptr));
  LOLA_CUDA_TRY(cudaMemcpy(host, tmp.p, count * c->ct_words() * 8, cudaMemcpyDeviceToHost));
  return LOLA_OK;
}

int lola_ct_import(lola_ctx* ctx, const uint64_t* host, size_t n_msg, lola_ct** out) {
  CHECK(ctx && out && (host || !n_msg), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  lola_ct* h = nullptr;
  TRY(new_ct(c, n_msg, &h));
  const size_t count = n_msg * c->kt;
  cudaError_t e = cudaMemcpy(h->ct.buf.p, host, count * c->ct_words() * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete h;
    return fail(LOLA_E_CUDA, cudaGetErrorString(e));
  }
  int rc = from_coeff(c, h->ct.buf.u64(), h->ct.buf.u64(), count, nullptr);
  if (rc == LOLA_OK && cudaDeviceSynchronize() != cudaSuccess) rc = fail(LOLA_E_CUDA, "import failed");
  if (rc != LOLA_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return LOLA_OK;
}

int lola_ct_copy_messages(lola_ctx* ctx, lola_ct* dst, size_t dst_off, const lola_ct* src, size_t src_off,
                          size_t n, void* stream) {
  CHECK(ctx && dst && src, LOLA_E_PARAM, "null argument");
  CHECK(dst_off + n <= dst->ct.n_msg && src_off + n <= src->ct.n_msg, LOLA_E_PARAM, "message range out of bounds");
  if (!n) return LOLA_OK;
  // a copy that overwrites all of dst takes src's level; otherwise the levels must agree
  if (dst_off == 0 && n == dst->ct.n_msg) dst->ct.level = src->ct.level;
  CHECK(dst->ct.L() == src->ct.L(), LOLA_E_PARAM, "ciphertexts of different levels");
  const size_t w = ctx->c->kt * 2 * (size_t)src->ct.L() * ctx->c->n;
  LOLA_CUDA_TRY(cudaMemcpyAsync(dst->ct.buf.u64() + dst_off * w, src->ct.buf.u64() + src_off * w, n * w * 8,
                                cudaMemcpyDeviceToDevice, to_stream(stream)));
  return LOLA_OK;
}

int lola_ct_upload(lola_ctx* ctx, lola_ct* ct, const uint64_t* host, void* stream) {
  CHECK(ctx && ct && host, LOLA_E_PARAM, "null argument");
  LOLA_CUDA_TRY(cudaMemcpyAsync(ct->ct.buf.p, host, ct->ct.used_words() * 8, cudaMemcpyHostToDevice, to_stream(stream)));
  return LOLA_OK;
}

int lola_ct_download(lola_ctx* ctx, const lola_ct* ct, uint64_t* host, void* stream) {
  CHECK(ctx && ct && host, LOLA_E_PARAM, "null argument");
  LOLA_CUDA_TRY(cudaMemcpyAsync(host, ct->ct.buf.p, ct->ct.used_words() * 8, cudaMemcpyDeviceToHost, to_stream(stream)));
  return LOLA_OK;
}

// ---------------------------------------------------------------- primitives
int lola_ntt_forward(lola_ctx* ctx, uint64_t* data, size_t n_polys, uint32_t n_limbs, void* stream) {
  CHECK(ctx && (data || !n_polys), LOLA_E_PARAM, "null argument");
  CHECK(n_limbs >= 1 && n_limbs <= ctx->c->L + ctx->c->K, LOLA_E_PARAM, "n_limbs out of range");
  return k::ntt_fwd(ctx->c, data, n_polys, n_limbs, 0, to_stream(stream));
}

int lola_ntt_inverse(lola_ctx* ctx, uint64_t* data, size_t n_polys, uint32_t n_limbs, void* stream) {
  CHECK(ctx && (data || !n_polys), LOLA_E_PARAM, "null argument");
  CHECK(n_limbs >= 1 && n_limbs <= ctx->c->L + ctx->c->K, LOLA_E_PARAM, "n_limbs out of range");
  return k::ntt_inv(ctx->c, data, n_polys, n_limbs, 0, false, to_stream(stream));
}

int lola_add(lola_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, void* stream) {
  CHECK(ctx && ((a && b && out) || !count), LOLA_E_PARAM, "null argument");
  return k::add(ctx->c, a, b, out, count, to_stream(stream));
}

int lola_rotate(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                const int32_t* steps, void* stream) {
  CHECK(ctx && keys && ((in && out && steps) || !count), LOLA_E_PARAM, "null argument");
  CHECK(in != out || !count, LOLA_E_PARAM, "rotation output must not alias its input");
  Ctx* c = ctx->c;
  if (!count) return LOLA_OK;
  cudaStream_t s = to_stream(stream);
  std::vector<uint32_t> g(count);
  std::vector<const uint64_t*> kp(count);
  for (size_t i = 0; i < count; ++i) {
    CHECK(steps[i] >= 0 && (uint32_t)steps[i] < c->n / 2, LOLA_E_PARAM, "rotation step out of range");
    g[i] = galois_for_step(c->n, steps[i]);
    const SwitchKey* key = keys->k->galois_key(g[i]);
    CHECK(key, LOLA_E_NOKEY, "missing Galois key for step " + std::to_string(steps[i]));
    kp[i] = key->buf.u64();
  }
  const size_t sw = rotate_scratch_words(c, count);
  void* buf = nullptr;
  const size_t bytes = sw * 8 + count * 16;
  LOLA_CUDA_TRY(cudaMallocAsync(&buf, bytes, s));
  uint64_t* scratch = (uint64_t*)buf;
  const uint64_t** dkeys = (const uint64_t**)(scratch + sw);
  uint32_t* dgal = (uint32_t*)(dkeys + count);
  int rc = LOLA_OK;
  if (cudaMemcpyAsync(dkeys, kp.data(), count * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dgal, g.data(), count * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(LOLA_E_CUDA, "upload of rotation tables failed");
  if (rc == LOLA_OK) {
    RotSpec rs;
    rs.d_gal = dgal;
    rs.d_keys = dkeys;
    rs.div = 1;
    rc = rotate(c, in, out, nullptr, count, rs, scratch, s);
  }
  // the host vectors above must outlive the async copies
  cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  return rc;
}

int lola_rotate_hoisted(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                        const int32_t* steps, size_t n_steps, void* stream) {
  CHECK(ctx && keys && ((in && out && steps) || !count || !n_steps), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  if (!count || !n_steps) return LOLA_OK;
  const size_t ctb = c->ct_words() * 8;
  CHECK((const char*)out + n_steps * count * ctb <= (const char*)in || (const char*)in + count * ctb <= (const char*)out,
        LOLA_E_PARAM, "rotation output must not overlap its input");
  CHECK(n_steps * count < (1ull << 32), LOLA_E_PARAM, "too many rotations in one call");
  cudaStream_t s = to_stream(stream);
  std::vector<uint32_t> g(n_steps);
  std::vector<const uint64_t*> kp(n_steps);
  for (size_t i = 0; i < n_steps; ++i) {
    CHECK(steps[i] >= 0 && (uint32_t)steps[i] < c->n / 2, LOLA_E_PARAM, "rotation step out of range");
    g[i] = galois_for_step(c->n, steps[i]);
    const SwitchKey* key = keys->k->galois_key(g[i]);
    CHECK(key, LOLA_E_NOKEY, "missing Galois key for step " + std::to_string(steps[i]));
    kp[i] = key->buf.u64();
  }
  const size_t sw = rotate_hoisted_scratch_words(c, count, n_steps);
  void* buf = nullptr;
  LOLA_CUDA_TRY(cudaMallocAsync(&buf, sw * 8 + n_steps * 16, s));
  uint64_t* scratch = (uint64_t*)buf;
  const uint64_t** dkeys = (const uint64_t**)(scratch + sw);
  uint32_t* dgal = (uint32_t*)(dkeys + n_steps);
  int rc = LOLA_OK;
  if (cudaMemcpyAsync(dkeys, kp.data(), n_steps * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dgal, g.data(), n_steps * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(LOLA_E_CUDA, "upload of rotation tables failed");
  if (rc == LOLA_OK) rc = rotate_hoisted(c, in, out, count, n_steps, dgal, dkeys, scratch, s);
  // the host vectors above must outlive the async copies
  cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  return rc;
}

int lola_rotate_sum(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out, size_t count,
                    const int32_t* steps, size_t n_steps, void* stream) {
  CHECK(ctx && keys && ((in && out && (steps || !n_steps)) || !count), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  if (!count) return LOLA_OK;
  const size_t ctb = c->ct_words() * 8;
  CHECK((const char*)out + count * ctb <= (const char*)in || (const char*)in + count * ctb <= (const char*)out,
        LOLA_E_PARAM, "rotate-sum output must not overlap its input");
  CHECK(n_steps <= 64, LOLA_E_PARAM, "at most 64 steps per rotate-sum");
  cudaStream_t s = to_stream(stream);
  std::vector<uint32_t> g(n_steps);
  std::vector<const uint64_t*> kp(n_steps);
  for (size_t i = 0; i < n_steps; ++i) {
    CHECK(steps[i] >= 0 && (uint32_t)steps[i] < c->n / 2, LOLA_E_PARAM, "rotation step out of range");
    g[i] = galois_for_step(c->n, steps[i]);
    const SwitchKey* key = keys->k->galois_key(g[i]);
    CHECK(key, LOLA_E_NOKEY, "missing Galois key for step " + std::to_string(steps[i]));
    kp[i] = key->buf.u64();
  }
  const size_t sw = rotate_sum_scratch_words(c, count);
  void* buf = nullptr;
  LOLA_CUDA_TRY(cudaMallocAsync(&buf, sw * 8 + n_steps * 16, s));
  uint64_t* scratch = (uint64_t*)buf;
  const uint64_t** dkeys = (const uint64_t**)(scratch + sw);
  uint32_t* dgal = (uint32_t*)(dkeys + n_steps);
  int rc = LOLA_OK;
  if (n_steps && (cudaMemcpyAsync(dkeys, kp.data(), n_steps * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                  cudaMemcpyAsync(dgal, g.data(), n_steps * 4, cudaMemcpyHostToDevice, s) != cudaSuccess))
    rc = fail(LOLA_E_CUDA, "upload of rotation tables failed");
  if (rc == LOLA_OK) rc = rotate_sum(c, in, out, count, (uint32_t)n_steps, dgal, dkeys, (uint32_t)count, scratch, s);
  // the host vectors above must outlive the async copies
  cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  return rc;
}

int lola_mod_switch(lola_ctx* ctx, const uint64_t* in, uint64_t* out, size_t count, uint32_t L_from, uint32_t L_to,
                    void* stream) {
  CHECK(ctx && ((in && out) || !count), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  CHECK(L_to >= 1 && L_to <= L_from && L_from <= c->L, LOLA_E_PARAM, "levels must satisfy 1 <= L_to <= L_from <= L");
  if (!count) return LOLA_OK;
  const size_t n = c->n;
  const char *ib = (const char*)in, *ob = (const char*)out;
  CHECK(ob + count * 2 * L_to * n * 8 <= ib || ib + count * 2 * L_from * n * 8 <= ob, LOLA_E_PARAM,
        "output must not overlap the input");
  cudaStream_t s = to_stream(stream);
  const size_t sw = mod_switch_scratch_words(c, count, L_from, L_to);
  void* buf = nullptr;
  if (sw) LOLA_CUDA_TRY(cudaMallocAsync(&buf, sw * 8, s));
  const int rc = mod_switch(c, in, out, count, L_from, L_to, (uint64_t*)buf, s);
  if (buf) cudaFreeAsync(buf, s);
  return rc;
}

int lola_autotune(lola_ctx* ctx, void* stream) {
  CHECK(ctx, LOLA_E_PARAM, "null argument");
  LOLA_CUDA_TRY(cudaSetDevice(ctx->c->device));
  return autotune(ctx->c, to_stream(stream));
}

int lola_tune_get(const lola_ctx* ctx, uint8_t* table, float* us) {
  CHECK(ctx && table, LOLA_E_PARAM, "null argument");
  const Tune& t = ctx->c->tune;
  CHECK(t.on, LOLA_E_STATE, "no tuning table installed");
  memcpy(table, t.v, sizeof(t.v));
  if (us) memcpy(us, t.us, sizeof(t.us));
  return LOLA_OK;
}

int lola_tune_set(lola_ctx* ctx, const uint8_t* table) {
  CHECK(ctx, LOLA_E_PARAM, "null argument");
  Tune t;
  if (table) {
    for (int i = 0; i < TUNE_KERNELS * TUNE_BUCKETS; ++i) {
      CHECK(table[i] < TV_COUNT, LOLA_E_PARAM, "tuning entry out of range");
      CHECK(table[i] == TV_CTA || ctx->c->logn == 14, LOLA_E_PARAM, "cluster geometries exist at n = 16384 only");
    }
    memcpy(t.v, table, sizeof(t.v));
    t.on = true;
  }
  ctx->c->tune = t;
  return LOLA_OK;
}

int lola_multiply(lola_ctx* ctx, const lola_keys* keys, const uint64_t* a, const uint64_t* b, uint64_t* out,
                  size_t count, const uint32_t* t_index, void* stream) {
  CHECK(ctx && keys && ((a && b && out) || !count), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  if (!count) return LOLA_OK;
  CHECK(out != a && out != b, LOLA_E_PARAM, "output must not alias an input");
  CHECK(keys->k->ev->relin, LOLA_E_NOKEY, "no relinearisation key");
  cudaStream_t s = to_stream(stream);
  std::vector<uint32_t> ti(count, 0);
  if (t_index)
    for (size_t i = 0; i < count; ++i) {
      CHECK(t_index[i] < c->kt, LOLA_E_PARAM, "t_index out of range");
      ti[i] = t_index[i];
    }
  const size_t sw = multiply_scratch_words(c, count, a == b);
  void* buf = nullptr;
  LOLA_CUDA_TRY(cudaMallocAsync(&buf, sw * 8 + count * 4, s));
  uint32_t* dti = (uint32_t*)((uint64_t*)buf + sw);
  int rc = LOLA_OK;
  if (cudaMemcpyAsync(dti, ti.data(), count * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(LOLA_E_CUDA, "upload failed");
  if (rc == LOLA_OK) rc = multiply(c, a, b, out, count, dti, 1, keys->k->ev->relin->buf.u64(), (uint64_t*)buf, s);
  cudaStreamSynchronize(s);
  cudaFreeAsync(buf, s);
  return rc;
}

int lola_mul_plain(lola_ctx* ctx, const uint64_t* in, const int64_t* slots, uint64_t* out, size_t count,
                   const uint32_t* t_index, void* stream) {
  CHECK(ctx && ((in && slots && out) || !count), LOLA_E_PARAM, "null argument");
  Ctx* c = ctx->c;
  if (!count) return LOLA_OK;
  cudaStream_t s = to_stream(stream);
  std::vector<uint32_t> ti(count, 0);
  if (t_index)
    for (size_t i = 0; i < count; ++i) {
      CHECK(t_index[i] < c->kt, LOLA_E_PARAM, "t_index out of range");
      ti[i] = t_index[i];
    }
  DevBuf pt;
  TRY(pt.alloc(count * c->L * c->n * 8));
  TRY(encode_plaintexts(c, slots, ti.data(), count, pt.u64(), s));
  // one ciphertext per launch-row: out_i = in_i (.) pt_i ; the multi kernel
  // indexes plaintexts as [r][t], so feed it one ciphertext at a time with kt = 1 views
  const size_t ctw = c->ct_words(), pw = (size_t)c->L * c->n;
  for (size_t i = 0; i < count; ++i) {
    // mul_plain_multi expects [B][kt] inputs and [R][kt] plaintexts; use the
    // element-wise Montgomery product on the two polynomials instead
    PrimeMap qm{};
    for (uint32_t l = 0; l < c->L; ++l) qm.p[l] = (uint8_t)l;
    TRY(k::axpy_mont_map(c, nullptr, in + i * ctw, pt.u64() + i * pw, out + i * ctw, c->L, c->L, qm, s));
    TRY(k::axpy_mont_map(c, nullptr, in + i * ctw + pw, pt.u64() + i * pw, out + i * ctw + pw, c->L, c->L, qm, s));
  }
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  return LOLA_OK;
}

// ------------------------------------------------------------------- networks
int lola_net_create(lola_ctx* ctx, const lola_input* input, const lola_layer* layers, size_t n_layers,
                    lola_net** out) {
  CHECK(ctx && out, LOLA_E_PARAM, "null argument");
  Net* n = nullptr;
  TRY(net_create(ctx->c, input, layers, n_layers, &n));
  *out = new lola_net{n, ctx};
  return LOLA_OK;
}

void lola_net_destroy(lola_net* net) {
  if (!net) return;
  delete net->net;
  delete net;
}

int lola_net_rotation_steps(const lola_net* net, int32_t* steps, size_t* count) {
  CHECK(net && count, LOLA_E_PARAM, "null argument");
  const auto& v = net->net->steps_needed;
  if (steps) std::copy(v.begin(), v.end(), steps);
  *count = v.size();
  return LOLA_OK;
}

int lola_net_output_map(const lola_net* net, uint32_t* msg, uint32_t* slot, size_t* count) {
  CHECK(net && count, LOLA_E_PARAM, "null argument");
  const auto& m = net->net->out_msg;
  if (msg) std::copy(m.begin(), m.end(), msg);
  if (slot) std::copy(net->net->out_slot.begin(), net->net->out_slot.end(), slot);
  *count = m.size();
  return LOLA_OK;
}

int lola_net_shape(const lola_net* net, uint32_t* in_msgs, uint32_t* out_msgs) {
  CHECK(net, LOLA_E_PARAM, "null argument");
  if (in_msgs) *in_msgs = net->net->n_in;
  if (out_msgs) *out_msgs = net->net->n_out;
  return LOLA_OK;
}

static int eval_impl(lola_ctx* ctx, const lola_keys* keys, lola_net* net, const lola_ct* in, lola_ct* out,
                     void* stream, bool graph) {
  CHECK(ctx && keys && net && in && out, LOLA_E_PARAM, "null argument");
  CHECK(net->net->ctx == ctx->c, LOLA_E_PARAM, "network belongs to another context");
  CHECK(in->ct.L() == ctx->c->L, LOLA_E_PARAM, "network input must be at the full level");
  CHECK(in != out, LOLA_E_PARAM, "input and output must differ");
  TRY(net_eval(ctx->c, keys->k, net->net, in->ct.buf.u64(), in->ct.n_msg, out->ct.buf.u64(), out->ct.n_msg,
               to_stream(stream), graph));
  out->ct.level = net->net->out_level == ctx->c->L ? 0 : net->net->out_level;
  return LOLA_OK;
}

int lola_eval_network(lola_ctx* ctx, const lola_keys* keys, lola_net* net, const lola_ct* in, lola_ct* out,
                      void* stream) {
  return eval_impl(ctx, keys, net, in, out, stream, true);
}

int lola_eval_network_eager(lola_ctx* ctx, const lola_keys* keys, lola_net* net, const lola_ct* in, lola_ct* out,
                            void* stream) {
  return eval_impl(ctx, keys, net, in, out, stream, false);
}

// ------------------------------------------------------------------ packing
int lola_pack_convolution(const int64_t* image, uint32_t h, uint32_t w, uint32_t kh, uint32_t kw, uint32_t s,
                          uint32_t n, int64_t* out, uint32_t* windows_out) {
  CHECK(image && out && kh && kw && s && kh <= h && kw <= w, LOLA_E_PARAM, "bad convolution shape");
  const uint32_t oh = (h - kh + s - 1) / s + 1, ow = (w - kw + s - 1) / s + 1;
  CHECK((uint64_t)oh * ow <= n, LOLA_E_PARAM, "too many windows for one message");
  memset(out, 0, sizeof(int64_t) * (size_t)kh * kw * n);
  for (uint32_t dr = 0; dr < kh; ++dr)
    for (uint32_t dc = 0; dc < kw; ++dc) {
      int64_t* msg = out + (size_t)(dr * kw + dc) * n;
      for (uint32_t i = 0; i < oh; ++i)
        for (uint32_t j = 0; j < ow; ++j) {
          const uint32_t r = s * i + dr, c = s * j + dc;
          msg[i * ow + j] = (r < h && c < w) ? image[(size_t)r * w + c] : 0;
        }
    }
  if (windows_out) *windows_out = oh * ow;
  return LOLA_OK;
}

int lola_pack_stacked(const int64_t* vec, uint32_t k, uint32_t d, uint32_t copies, uint32_t n, int64_t* out) {
  CHECK(vec && out && d < 31 && k <= (1u << d) && (uint64_t)copies << d <= n, LOLA_E_PARAM, "bad stacked shape");
  memset(out, 0, sizeof(int64_t) * n);
  for (uint32_t b = 0; b < copies; ++b)
    for (uint32_t i = 0; i < k; ++i) out[((size_t)b << d) + i] = vec[i];
  return LOLA_OK;
}

// ---------------------------------------------------------------- profiling
int lola_profile_enable(lola_ctx* ctx, int kind, int on) {
  CHECK(ctx, LOLA_E_PARAM, "null context");
  return profile_enable(ctx->c, kind, on);
}

int lola_profile_read(lola_ctx* ctx, int kind, double* ms, uint64_t* launches, uint64_t* units) {
  CHECK(ctx, LOLA_E_PARAM, "null context");
  return profile_read(ctx->c, kind, ms, launches, units);
}

int lola_profile_kinds(void) { return KI_COUNT; }
const char* lola_profile_name(int kind) { return kernel_name(kind); }

uint64_t lola_launch_count(const lola_ctx* ctx) { return ctx ? ctx->c->launches.load() : 0; }

int lola_alu_rate(lola_ctx* ctx, int kind, double* per_second, double* ms) {
  CHECK(ctx, LOLA_E_PARAM, "null context");
  return alu_rate(ctx->c, kind, per_second, ms);
}

}  // extern "C"
