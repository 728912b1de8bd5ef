// Autotuning of the key-switch transforms' launch geometry (decompose,
// mod-up, INTT mod P, mod-down; one CTA per limb, or at n = 16384 a 2-CTA
// cluster per limb with 16 or 32 words per thread or a 4-CTA cluster with 16)
// per launch-size bucket.
//
// What is timed is the chain the geometry serves: whole rotations (decompose
// -> mod-up -> inner product -> INTT mod P -> mod-down) of 1, 4, 16, 64 and
// 256 ciphertexts on zero-filled buffers with a zero key, with CUDA events
// around runs of back-to-back rotations (best of three runs).  For each
// ciphertext count and each kernel, the table entry of the bucket that
// kernel's launch falls in is set to every geometry in turn (coordinate
// descent, smallest counts first; an entry is decided by the first count
// that reaches it), and a geometry replaces the library's default only when
// the rotations get faster by more than kMargin: timings of isolated runs
// carry a few percent of noise.  The variants compute the same words, so
// the choice changes time only.
#include <algorithm>

#include "he.h"

namespace lola {

int tune_bucket(size_t units) {
  int b = 0;
  for (size_t u = 64; b < TUNE_BUCKETS - 1 && units >= u; u *= 4) ++b;
  return b;
}

static const size_t kCounts[] = {1, 4, 16, 64, 256};
static constexpr size_t kMaxCts = 256;
static constexpr float kMargin = 0.03f;

// microseconds per rotation of `count` ciphertexts with the current table
static int time_rotations(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, const RotSpec& rs,
                          uint64_t* scratch, cudaStream_t s, float* us) {
  int rc = LOLA_OK;
  for (int r = 0; r < 2 && rc == LOLA_OK; ++r) rc = rotate(c, in, out, nullptr, count, rs, scratch, s);   // warm-up
  if (rc != LOLA_OK) return rc;
  cudaEvent_t e0, e1;
  LOLA_CUDA_TRY(cudaEventCreate(&e0));
  LOLA_CUDA_TRY(cudaEventCreate(&e1));
  constexpr int reps = 6, trials = 3;
  float best = 0;
  cudaError_t e = cudaSuccess;
  for (int tr = 0; tr < trials && rc == LOLA_OK && e == cudaSuccess; ++tr) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && rc == LOLA_OK; ++r) rc = rotate(c, in, out, nullptr, count, rs, scratch, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (tr == 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LOLA_OK) return rc;
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
  *us = best * 1000.0f / reps;
  return LOLA_OK;
}

int autotune(Ctx* c0, cudaStream_t s) {
  Ctx* c = c0->root;
  const size_t n = c->n, L = c->L, LK = c->L + c->K;
  Tune t;
  t.on = true;
  const size_t per[TUNE_KERNELS] = {L, c->host.mu_n[1], 2 * (size_t)c->K, 2 * L};
  // start from the defaults (the table then reproduces them exactly where
  // nothing is measured faster)
  for (int kern = 0; kern < TUNE_KERNELS; ++kern)
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
      const size_t lo = b == 0 ? 1 : (size_t)16 << (2 * b);   // smallest launch of the bucket
      t.v[kern][b] = (uint8_t)k::default_geometry(c, kern, lo);
    }
  const int nvar = c->logn == 14 ? (int)TV_COUNT : 1;   // cluster variants exist at n = 16384
  if (nvar == 1 || !c->K) {                                // nothing to choose
    c->tune = t;
    return LOLA_OK;
  }
  // buffers: input and output ciphertexts, rotation scratch, a zero key
  const size_t w_ct = kMaxCts * c->ct_words(), w_scr = rotate_scratch_words(c, kMaxCts), w_key = 2 * c->dnum * LK * n;
  const size_t words = 2 * w_ct + w_scr + w_key;
  void* buf = nullptr;
  LOLA_CUDA_TRY(cudaMallocAsync(&buf, words * 8, s));
  uint64_t* in = (uint64_t*)buf;
  uint64_t* out = in + w_ct;
  uint64_t* scratch = out + w_ct;
  uint64_t* key = scratch + w_scr;
  int rc = LOLA_OK;
  if (cudaMemsetAsync(buf, 0, words * 8, s) != cudaSuccess) rc = fail(LOLA_E_CUDA, "autotune: memset failed");
  RotSpec rs;
  rs.gal = galois_for_step(c->n, 1);
  rs.key = key;
  const Tune saved = c->tune;
  bool decided[TUNE_KERNELS][TUNE_BUCKETS] = {};
  for (size_t count : kCounts) {
    for (int kern = 0; kern < TUNE_KERNELS && rc == LOLA_OK; ++kern) {
      const int b = tune_bucket(count * per[kern]);
      if (decided[kern][b]) continue;
      decided[kern][b] = true;
      const int d = t.v[kern][b];
      float us[TV_COUNT] = {};
      for (int v = 0; v < nvar && rc == LOLA_OK; ++v) {
        t.v[kern][b] = (uint8_t)v;
        c->tune = t;
        rc = time_rotations(c, in, out, count, rs, scratch, s, &us[v]);
      }
      if (rc != LOLA_OK) break;
      int pick = d;
      for (int v = 0; v < nvar; ++v)
        if (us[v] < us[pick] && us[v] < (1.0f - kMargin) * us[d]) pick = v;
      t.v[kern][b] = (uint8_t)pick;
      for (int v = 0; v < nvar; ++v) t.us[kern][b][v] = us[v];
    }
    if (rc != LOLA_OK) break;
  }
  cudaFreeAsync(buf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LOLA_OK) rc = fail(LOLA_E_CUDA, "autotune failed");
  c->tune = rc == LOLA_OK ? t : saved;
  return rc;
}

}  // namespace lola
