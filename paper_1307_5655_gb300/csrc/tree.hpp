// Internal representation of a compiled evaluation tree and of the flattened
// per-point schedule the kernels replay.  Not part of the C ABI.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <vector_types.h>

#include "../../include/fastpoly.h"

namespace fp {

// Schedule control word of one non-root node, in node index order (Sec. 1):
//   bits  0..5   S     lazy height of the node (its accumulator slot)
//   bits  6..11  D     lazy height of its parent (the slot it feeds)
//   bit  12      LEAF  the node has no children
//   bit  13      FIRST the node is the lowest-index child of its parent
//   bits 14..31  PID   index of x_v^d in the per-point power table
constexpr uint32_t kCtrlS = 0, kCtrlD = 6, kCtrlLeaf = 12, kCtrlFirst = 13, kCtrlPid = 14;
constexpr uint32_t kMaxPowers = 1u << 15;

// Power program entry, one per power-table slot, in dependency order:
//   bits  0..1   op   0: load x_v (A1 = v)   1: square of slot A1
//                     2: slot A1 times slot A2 (A2 holds x_v)
//   bits  2..16  A1
//   bits 17..31  A2
constexpr uint32_t kPowLoad = 0, kPowSq = 1, kPowMulX = 2;

// Ops for the fused value types (FP64, FP32C, MODP): the walk grouped into
// ops, each ending with the outgoing multiply-add of its last node.  One op
// record (32 bytes, read with two 128-bit loads) per op:
//   x: bits 0..1 kind  (0: one node; 1: chain j0..j0+len-1, each node the only
//                       child of the next; 2: dense subtree block of len nodes
//                       evaluated by the scheme's own splits in registers;
//                       3: partial block -- the last node N of the run and its
//                       last children, which together are the lower part b of
//                       a split p = a x^f + b of N's own run (Def. 1.2): b is
//                       evaluated like a block, with N's slot S (c_N plus
//                       N's earlier, larger children) as the value of N)
//      bits 2..7 S, 8..13 D, 14 LEAF (first node of the op is a leaf),
//      15 FIRST (last node is its parent's first child), 16 UNIFORM (all
//      powers inside a chain are the same), 17..31 PID of the outgoing edge
//   y: bits 0..7 len - 1; for a block or partial block of more than
//      kMaxBlock nodes, bits 8..15 f = the scheme's split of the run and
//      bits 16..31 the table position of x^f: the run is T(b) + T(a) x^f,
//      b its f lowest nodes, and its coefficients are stored as two runs
//      (a, then b), each from a multiple of 4 elements
//   z: first node j0      w: offset of the op's coefficients (bits 0..30);
//      bit 31: the op lies past the split and its edge goes into the root's
//      slot (see ops_layout)
//   a: leaf coefficient of a single-node op   b: parent coefficient if FIRST
// The coefficients of chains and blocks are stored per op in a stream, each
// op's run starting at a multiple of 4 elements (aligned vector loads).
constexpr uint32_t kOpNode = 0, kOpChain = 1, kOpBlock = 2, kOpPartial = 3;
constexpr uint32_t kOpS = 2, kOpD = 8, kOpLeaf = 14, kOpFirst = 15, kOpUniform = 16, kOpPid = 17;
constexpr int kMaxChain = 64, kMaxBlock = 16, kStreamAlign = 4;
// a floating-point block of kMaxBlock < len <= kMaxSplitBlock nodes runs as
// its two parts T(run) = T(b) + T(a) x^f, each at most kMaxBlock nodes
constexpr int kMaxSplitBlock = 2 * kMaxBlock;
constexpr int kMaxTwoPartBlock = 22;  // the longest run the compiler forms into two parts
// PID of a block or partial block of a Balanced tree whose edge power is not
// in the table: the
// op recomputes x_b^d from a kept power x_b^(d >> m) (or x_b itself), its
// record's z = base position (bits 0..14; 0x7FFF: x_b) | m << 15 (4 bits) |
// (d mod 2^m) << 19, with the power program's steps (square, times x_b)
constexpr uint32_t kPidRecompute = 0x7FFFu;
constexpr int kRecomputeMinEntries = 20;  // only tables of at least this many entries per point shrink
constexpr int kRecomputeCost = 16;        // ops x steps per point a recomputed power may cost
constexpr int kRecomputeMaxSteps = 13;
constexpr int kMaxExactBlock = 64;  // blocks of mod-p trees (evaluated by a loop, not a template)

template <class C>
struct alignas(16) OpRec {
  uint32_t x, y, z, w;
  C a, b;
};

struct DeviceSchedule {
  int device = -1;
  uint32_t* ctrl = nullptr;   // [nsteps]
  uint32_t* pow_prog = nullptr;  // [npow]
  uint2* pow_dv = nullptr;       // [npow] (variable, degree)
  double* ca_f64 = nullptr;   // [nsteps] coefficient of the node
  double* cb_f64 = nullptr;   // [nsteps] coefficient of the parent when FIRST, else 0
  float* ca_f32 = nullptr;
  float* cb_f32 = nullptr;
  uint64_t* ca_u64 = nullptr;
  uint64_t* cb_u64 = nullptr;
  OpRec<double>* ops_f64 = nullptr;  // [nops]
  OpRec<float>* ops_f32 = nullptr;
  OpRec<uint64_t>* ops_u64 = nullptr;
  double* st_f64 = nullptr;          // coefficient stream of chains and blocks
  float* st_f32 = nullptr;
  uint64_t* st_u64 = nullptr;
  uint2* ops_prog = nullptr;         // power program of the grouped-op kernel
  uint32_t* ops_chain_pid = nullptr;  // [nsteps]
  uint2* ops_defer = nullptr;         // [ops_ndefer] edges into the root past the split
  // residues (fp_compile_rns), one slice per prime
  uint64_t* ca_rns = nullptr;        // [k][nsteps]
  uint64_t* cb_rns = nullptr;        // [k][nsteps]
  OpRec<uint64_t>* ops_rns = nullptr;  // [k][nops]
  uint64_t* st_rns = nullptr;        // [k][stream_pitch]
  uint64_t* root_rns = nullptr;      // [k]
  int64_t st_rns_pitch = 0;
};

}  // namespace fp

struct fp_tree {
  int nvars = 1;
  int coeff_type = FP_F64;  // FP_F64 or FP_MODP
  int64_t nnodes = 0;       // 0: the zero polynomial
  int64_t nterms_in = 0;    // terms given to fp_compile (term_of_node indexes them)
  std::vector<int32_t> node_e;       // [nnodes][nvars]
  std::vector<int64_t> term_of_node;  // -1: virtual group root
  std::vector<int64_t> parent;       // -1: root
  std::vector<int32_t> pd_var;
  std::vector<int64_t> pd;
  std::vector<int32_t> lh;
  std::vector<double> c_f64;    // node coefficients (coeff_type FP_F64)
  std::vector<uint64_t> c_u64;  // node coefficients (coeff_type FP_MODP)
  int max_lh = 0;

  // flattened schedule
  std::vector<uint32_t> ctrl;      // [nnodes-1]
  std::vector<uint32_t> pow_prog;  // [npow]
  std::vector<int32_t> pow_var;
  std::vector<int64_t> pow_deg;
  int root_leaf = 1;
  int root_lh = 0;
  int root_pid = -1;

  // grouped ops for the fused value types
  std::vector<uint4> ops;          // x, y, z, w of each op record
  std::vector<int64_t> op_a_node;  // node whose coefficient is the op's leaf value, or -1
  std::vector<int64_t> op_b_node;  // parent whose coefficient initialises the slot, or -1
  std::vector<int64_t> stream;     // node whose coefficient sits at each stream slot, or -1 (padding)
  int block_scheme = 0;            // FP_SCHEME_E or FP_SCHEME_B when blocks are used, else 0
  int pid_x1 = -1;                 // power slot of x_b, b = the innermost variable (blocks run over it)
  int pid_pow[fp::kMaxBlock + 1] = {};  // power slot of x_b^d, d <= kMaxBlock (-1: absent)

  // the grouped-op kernel's per-point table: the walk's powers at positions
  // [0, ops_nlive), its slots at [ops_nlive, ops_nlive + ops_nslot); the op
  // records above carry slots and powers in this layout
  std::vector<uint2> ops_prog;          // {op | A1 << 2 | A2 << 17 (positions), destination}
  std::vector<uint32_t> ops_chain_pid;  // [nnodes-1] position of each node's edge power
  int ops_nlive = 0, ops_nslot = 1, ops_entries = 1;
  int ops_root_lh = 0, ops_root_pid = -1;
  int ops_pos_x1 = -1;  // position of x_b when the walk reads it
  int ops_ext = 0;      // two-part blocks or recomputed edge powers (Balanced)
  int64_t ops_split = 0;  // first op of the root's later children (0: no split; see ops_layout)
  int ops_ndefer = 0;     // ops from ops_split on whose edge goes into the root's slot
  std::vector<uint2> ops_defer;  // those ops' {PID, z} in walk order (their edge powers)
  int ops_pid_pow[fp::kMaxBlock + 1] = {};  // position of x_b^d for the block templates (-1: absent)

  // residue number system (fp_compile_rns): coefficients modulo rns_k primes,
  // [rns_k][nnodes]; coeff_type is then FP_RNS_COEFFS
  int rns_k = 0;
  std::vector<uint64_t> c_rns;

  // launch configuration chosen by fp_tune per value type (kernel, ppt; 0 = not tuned)
  int tuned_kernel[4] = {0, 0, 0, 0};
  int tuned_ppt[4] = {0, 0, 0, 0};

  fp::DeviceSchedule dev;
};

namespace fp {
// Stream-ordered work space from the library's device pool (freed with
// cudaFreeAsync; the pool keeps freed memory mapped for reuse).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);

// Build the tree and its schedule on the host (no CUDA calls).
int compile_host(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs,
                 fp_dtype coeff_type, fp_scheme scheme, const int32_t* f_table,
                 int64_t f_table_len, fp_tree* t);

// Bounds check of a compiled schedule against the arrays and tables the
// kernels index: FP_OK, or FP_E_INTERNAL (compile_host ends with it).
int validate_schedule(const fp_tree* t);
}  // namespace fp
