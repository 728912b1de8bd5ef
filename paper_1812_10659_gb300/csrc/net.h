// LoLa network: layer list -> op list over message registers -> executor.
#pragma once
#include <map>
#include <memory>
#include <vector>

#include "he.h"

namespace lola {

enum OpKind {
  OP_MAC = 1, OP_ROT = 2, OP_SUM = 3, OP_MULPT = 4, OP_SQUARE = 5, OP_ROT_HOISTED = 6, OP_MODSWITCH = 7,
  OP_ROT_SUM = 8
};

// A register holds `msgs` messages for every request of the batch and every
// plaintext modulus: layout [msg][request][t_i][2][L'][n], L' the register's
// level (ciphertext primes left after modulus switching).
struct Op {
  OpKind kind;
  int dst = -1, src = -1, aux = -1;   // virtual registers
  uint32_t dst_off = 0, src_off = 0, aux_off = 0;
  uint32_t msgs = 0;                  // messages processed
  uint32_t level = 0;                 // ciphertext primes of the operands
  uint32_t level_to = 0;              // OP_MODSWITCH: primes of the result
  // OP_ROT: per-message rotation step (0 = row swap); aux = accumulator register (or -1)
  // OP_ROT_HOISTED: message src_off of src rotated by steps[m] into message m of dst
  // OP_ROT_SUM: message m of src plus its rotations by every one of steps
  // (the same steps for all messages) into message m of dst, one key switch
  std::vector<int32_t> steps;
  // OP_MULPT: plaintexts [msgs][kt][level][n] at pt_first (in plaintext blocks
  // of the op's level); src_stride 0 = broadcast
  size_t pt_first = 0;
  uint32_t src_stride = 1;
  // OP_MAC: R inputs per output, weight table offset (entries [R][kt][L][msgs])
  uint32_t R = 0;
  size_t w_first = 0;
  // OP_SUM: dst = sum of `msgs` messages of src (+ message aux_off of aux if aux >= 0)
};

struct Net {
  Ctx* ctx = nullptr;
  uint32_t n_in = 0, n_out = 0;
  std::vector<uint32_t> vreg_msgs;    // size of each virtual register (messages)
  std::vector<uint32_t> vreg_level;   // its level (ciphertext primes)
  std::map<uint32_t, Ctx*> lctx;      // level -> context (owned by the root context)
  uint32_t out_level = 0;
  int in_reg = -1, out_reg = -1;
  std::vector<Op> ops;
  std::vector<uint32_t> out_msg, out_slot;
  std::vector<int32_t> steps_needed;  // distinct rotation steps (0 = row swap)
  bool needs_relin = false;
  std::map<uint32_t, DevBuf> pt;      // level -> encoded plaintexts [blocks][kt][level][n]
  DevBuf w, ws;                       // MAC scalars and Shoup companions
  std::map<uint32_t, std::unique_ptr<struct Executor>> exec;   // by batch size
  ~Net();
};

int net_create(Ctx* c, const lola_input* in, const lola_layer* layers, size_t n_layers, Net** out);
int net_eval(Ctx* c, const KeySet* ks, Net* net, const uint64_t* d_in, size_t in_msgs, uint64_t* d_out,
             size_t out_msgs, cudaStream_t s, bool use_graph);

}  // namespace lola
