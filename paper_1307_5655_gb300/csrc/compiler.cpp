// Host compiler: terms -> evaluation tree -> flattened per-point schedule.
//
// Follows Moroz, "Fast polynomial evaluation and composition":
//   Sec. 1 (decreasing lex order <_t, root = last node), Def. 1.1 (partial
//   degrees), Def. 1.2 (function scheme split p = a x^f(n) + b with b the
//   f(n) lowest terms, n = #terms - 1), the Remark on multivariate polynomials
//   (the scheme applied per variable: terms grouped by the first variable's
//   exponent, each group compiled over the next variable and represented by
//   its lowest term; a group missing that term gets a zero-coefficient root),
//   Def. 1.3 (lazy height, with the first-walked child counted:
//   lh(N) = max(lh(C1), 1 + max_{i>=2} lh(Ci))), Sec. 2.2 (distinct powers,
//   computed once per point by squarings and multiplications by x).
#include <algorithm>
#include <cstring>
#include <map>
#include <new>

#include "tree.hpp"

namespace fp {
namespace {

// f(n) of a scheme; n = #terms - 1 >= 1.  Returns 0 when undefined.
int64_t split_count(fp_scheme s, const int32_t* ft, int64_t ftlen, int64_t n) {
  switch (s) {
    case FP_SCHEME_D: return n;
    case FP_SCHEME_H: return 1;
    case FP_SCHEME_E: {
      int64_t f = 1;
      while ((f << 1) <= n) f <<= 1;
      return f;
    }
    case FP_SCHEME_B: return (n + 1) >> 1;
    case FP_SCHEME_CUSTOM: return (ft && n < ftlen) ? ft[n] : 0;
  }
  return 0;
}

struct Builder {
  int nv;
  const std::vector<int32_t>& e;  // [N][nv]
  std::vector<int64_t>& parent;
  std::vector<int32_t>& pd_var;
  std::vector<int64_t>& pd;
  fp_scheme scheme;
  const int32_t* ft;
  int64_t ftlen;
  int status = FP_OK;

  int32_t ex(int64_t node, int v) const { return e[node * nv + v]; }

  // Attach the units (groups) of one level by the function scheme.
  void attach_units(const std::vector<int64_t>& root, int var) {
    std::vector<std::pair<int64_t, int64_t>> work;
    work.emplace_back(0, (int64_t)root.size() - 1);
    while (!work.empty() && status == FP_OK) {
      auto [a, b] = work.back();
      work.pop_back();
      if (a >= b) continue;
      const int64_t n = b - a;
      const int64_t f = split_count(scheme, ft, ftlen, n);
      if (f < 1 || f > n) { status = FP_E_BAD_SCHEME; return; }
      const int64_t top = root[b - f], base = root[b];  // roots of T_a and T_b
      parent[top] = base;
      pd_var[top] = var;
      pd[top] = (int64_t)ex(top, var) - ex(base, var);
      work.emplace_back(b - f + 1, b);  // b: the f lowest units
      work.emplace_back(a, b - f);      // a: the rest
    }
  }

  // Nodes [lo, hi] agree on the variables before `var`.
  void level(int64_t lo, int64_t hi, int var) {
    std::vector<int64_t> roots;
    int64_t start = lo;
    for (int64_t i = lo; i <= hi && status == FP_OK; ++i) {
      if (i == hi || ex(i, var) != ex(i + 1, var)) {
        if (var + 1 < nv) level(start, i, var + 1);
        roots.push_back(i);
        start = i + 1;
      }
    }
    if (status == FP_OK) attach_units(roots, var);
  }
};

// Emit the sorted terms of `run` (sharing their first `var` exponents) into
// `out`, appending a virtual node (prefix, 0, ..., 0) when the run lacks it.
void emit_with_roots(const std::vector<int64_t>& order, int64_t lo, int64_t hi, int var, int nv,
                     const int32_t* exps, std::vector<int32_t>& out_e, std::vector<int64_t>& out_t) {
  if (var == nv) {  // a single term
    out_e.insert(out_e.end(), exps + order[lo] * nv, exps + order[lo] * nv + nv);
    out_t.push_back(order[lo]);
    return;
  }
  int64_t start = lo;
  int32_t last_val = -1;
  for (int64_t i = lo; i <= hi; ++i) {
    const int32_t v = exps[order[i] * nv + var];
    if (i == hi || exps[order[i + 1] * nv + var] != v) {
      emit_with_roots(order, start, i, var + 1, nv, exps, out_e, out_t);
      last_val = v;
      start = i + 1;
    }
  }
  if (var > 0 && last_val != 0) {
    // the run's root (prefix, 0, ..., 0) is missing
    const int32_t* pre = exps + order[lo] * nv;
    for (int v = 0; v < nv; ++v) out_e.push_back(v < var ? pre[v] : 0);
    out_t.push_back(-1);
  }
}

// a6: the grouped-op kernel's own per-point table (shared memory is what
// bounds its occupancy).  The ops form a tree of their own: an op feeds the
// slot of its last node's parent and reads at most one slot (its first node's
// for a node or chain, its last node's for a partial block; none for a block
// or a run starting at a leaf).  Only nodes that ops feed own a slot, and the
// lazy-height rule of Def. 1.3 applied to that tree, with -1 for an op that
// reads no slot, numbers the slots: lh(N) = max(lh(C1), 1 + max_{i>=2} lh(Ci)).
// The table holds, at positions [0, nlive), the powers the walk reads (op
// edges, chain edges, the root's) and above them the slots; the power
// program writes explicit positions, so its temporaries and the powers only
// the block templates use (read into registers before the walk) live above
// nlive too, where the slots later reuse the space.
int ops_layout(fp_tree* t) {
  const int64_t N = t->nnodes;
  const size_t nops = t->ops.size();
  // op-tree lazy heights
  std::vector<int32_t> first_h(N, -1), rest_h(N, -2), olh(N, 0);
  std::vector<uint8_t> fed(N, 0), done(N, 0);
  auto finalize = [&](int64_t r) {
    if (!done[r]) {
      olh[r] = fed[r] ? std::max({first_h[r], rest_h[r] + 1, 0}) : 0;
      done[r] = 1;
    }
    return olh[r];
  };
  std::vector<int64_t> reads(nops, -1);
  for (size_t i = 0; i < nops; ++i) {
    const uint32_t x = t->ops[i].x, kind = x & 3u;
    const int64_t j0 = t->ops[i].z, j1 = j0 + (t->ops[i].y & 255u);
    const bool leaf = (x >> kOpLeaf) & 1u;
    if (kind == kOpPartial) reads[i] = j1;
    else if (kind != kOpBlock && !leaf) reads[i] = j0;
    const int32_t h = reads[i] >= 0 ? finalize(reads[i]) : -1;
    const int64_t q = t->parent[j1];
    if (!fed[q]) {
      fed[q] = 1;
      first_h[q] = h;
    } else {
      rest_h[q] = std::max(rest_h[q], h);
    }
  }
  const int32_t root_h = t->root_leaf ? 0 : finalize(N - 1);
  int32_t nslot = 1;
  for (int64_t r = 0; r < N; ++r)
    if (fed[r]) nslot = std::max(nslot, finalize(r) + 1);
  if (nslot - 1 > FP_MAX_LAZY_HEIGHT) return FP_E_TOO_LARGE;  // 6-bit slot fields

  // The split of the op list for small grids: the root's first child (the
  // upper part a of the top split p = a x^f + b) heads a subtree of nodes
  // 0 .. ra, and ops [0, s) cover exactly those nodes; ops [s, nops) add the
  // root's later children into its slot.  The two ranges can run in two
  // warps, the second applying its edges into the root's slot (marked below)
  // to the first's root slot afterwards, in walk order.  Kept when each range
  // has at least a quarter of the nodes.
  t->ops_split = 0;
  if (N > 2) {
    int64_t ra = -1;
    for (int64_t j = 0; j + 1 < N && ra < 0; ++j)
      if (t->parent[j] == N - 1) ra = j;
    std::vector<int64_t> sz(N, 1);
    for (int64_t j = 0; j + 1 < N; ++j) sz[t->parent[j]] += sz[j];
    if (ra >= 0 && ra - sz[ra] + 1 == 0 && 4 * (ra + 1) >= N && 4 * (N - 1 - ra) >= N)
      for (size_t i = 1; i < nops; ++i) {
        const int64_t prev_j1 = (int64_t)t->ops[i - 1].z + (t->ops[i - 1].y & 255u);
        if (prev_j1 == ra && (int64_t)t->ops[i].z == ra + 1) {
          t->ops_split = (int64_t)i;
          break;
        }
      }
  }
  // past the split, the edges into the root's slot are marked (w bit 31):
  // the second warp keeps their values and applies them after the first
  // warp's part, in walk order, so the split's result is the walk's own
  t->ops_ndefer = 0;
  if (t->ops_split > 0)
    for (size_t i = (size_t)t->ops_split; i < nops; ++i) {
      const int64_t j1 = (int64_t)t->ops[i].z + (t->ops[i].y & 255u);
      if (t->parent[j1] == N - 1) {
        t->ops[i].w |= 0x80000000u;
        ++t->ops_ndefer;
      }
    }

  // powers the walk reads, and the block templates' powers
  const size_t np = t->pow_prog.size();
  std::vector<uint8_t> live(np, 0), tmpl(np, 0), needed(np, 0);
  for (size_t i = 0; i < nops; ++i) {
    live[t->ops[i].x >> kOpPid] = 1;
    if ((t->ops[i].y >> 8) & 255u) live[t->ops[i].y >> 16] = 1;  // x^f of a two-part block
    if ((t->ops[i].x & 3u) == kOpChain)
      for (int64_t j = t->ops[i].z; j < (int64_t)t->ops[i].z + (t->ops[i].y & 255u); ++j)
        live[t->ctrl[j] >> kCtrlPid] = 1;
  }
  if (t->root_pid >= 0) live[t->root_pid] = 1;
  // Balanced trees: edge powers of the block variable that few ops read (the
  // top levels: one partial block reads x^5003) stay out of the table when
  // the table is large enough to bound the points resident per SM: the block
  // or partial block recomputes its edge power from the nearest binary prefix
  // x^(d >> m) that is kept, or from x itself (in registers), by the power
  // program's own steps, so the value is the same.  A power is recomputed
  // while its ops x steps stay within kRecomputeCost (prefixes are decided
  // first: powers in increasing degree).
  std::vector<uint8_t> rare(np, 0);
  std::vector<uint32_t> redge(np, 0);  // the recompute word of a rare power
  int32_t nlive0 = 0;
  for (size_t k = 0; k < np; ++k) nlive0 += live[k];
  if (t->block_scheme == FP_SCHEME_B && nlive0 + nslot >= kRecomputeMinEntries) {
    const int32_t bv = t->nvars - 1;
    std::vector<int64_t> uses(np, 0);
    std::vector<uint8_t> pinned(np, 0);  // read by chains, single nodes, joins or the root
    for (size_t i = 0; i < nops; ++i) {
      const uint32_t kind = t->ops[i].x & 3u, pid = t->ops[i].x >> kOpPid;
      if (kind == kOpBlock || kind == kOpPartial) uses[pid]++;
      else pinned[pid] = 1;
      if ((t->ops[i].y >> 8) & 255u) pinned[t->ops[i].y >> 16] = 1;
      if (kind == kOpChain)
        for (int64_t j = t->ops[i].z; j < (int64_t)t->ops[i].z + (t->ops[i].y & 255u); ++j)
          pinned[t->ctrl[j] >> kCtrlPid] = 1;
    }
    if (t->root_pid >= 0) pinned[t->root_pid] = 1;
    std::map<int64_t, size_t> of_deg;  // degree -> power id, block variable (increasing degree)
    for (size_t k = 0; k < np; ++k)
      if (t->pow_var[k] == bv) of_deg[t->pow_deg[k]] = k;
    for (const auto& [d, k] : of_deg) {
      if (!live[k] || pinned[k] || uses[k] == 0) continue;
      for (int m = 1; m <= kRecomputeMaxSteps && (d >> m) >= 1; ++m) {
        const int64_t b = d >> m;
        uint32_t base;
        if (b == 1) {
          base = 0x7FFFu;
        } else {
          const auto it = of_deg.find(b);
          if (it == of_deg.end() || !live[it->second] || rare[it->second]) continue;
          base = (uint32_t)it->second;  // a power id for now, its position below
        }
        if (uses[k] * m <= kRecomputeCost) {
          rare[k] = 1;
          redge[k] = base | (uint32_t)m << 15 | (uint32_t)(d & ((1ll << m) - 1)) << 19;
        }
        break;  // the nearest kept prefix decides
      }
    }
    for (size_t k = 0; k < np; ++k)
      if (rare[k]) live[k] = 0;
  }
  if (t->block_scheme)
    for (int d = 1; d <= kMaxBlock; ++d)
      if (t->pid_pow[d] >= 0) tmpl[t->pid_pow[d]] = 1;
  for (size_t k = 0; k < np; ++k) needed[k] = live[k] | tmpl[k];
  for (size_t k = np; k-- > 0;) {  // operands of needed powers (program order is dependency order)
    if (!needed[k]) continue;
    const uint32_t w = t->pow_prog[k], op = w & 3u;
    if (op == kPowSq || op == kPowMulX) needed[(w >> 2) & 0x7FFFu] = 1;
    if (op == kPowMulX) needed[w >> 17] = 1;
  }
  std::vector<int32_t> pos(np, -1);
  int32_t nlive = 0;
  for (size_t k = 0; k < np; ++k)
    if (live[k]) pos[k] = nlive++;
  std::vector<int64_t> last_use(np, -1);
  for (size_t k = 0; k < np; ++k) {
    if (!needed[k]) continue;
    const uint32_t w = t->pow_prog[k], op = w & 3u;
    if (op == kPowSq || op == kPowMulX) last_use[(w >> 2) & 0x7FFFu] = (int64_t)k;
    if (op == kPowMulX) last_use[w >> 17] = (int64_t)k;
  }
  std::vector<int32_t> free_pos;
  int32_t top = nlive;  // one past the highest position written
  t->ops_prog.clear();
  for (size_t k = 0; k < np; ++k) {
    if (!needed[k]) continue;
    if (pos[k] < 0) {
      if (!free_pos.empty()) {
        pos[k] = free_pos.back();
        free_pos.pop_back();
      } else {
        pos[k] = top++;
      }
    }
    const uint32_t w = t->pow_prog[k], op = w & 3u;
    uint32_t a1 = (w >> 2) & 0x7FFFu, a2 = w >> 17;
    if (op == kPowSq || op == kPowMulX) a1 = (uint32_t)pos[a1];
    if (op == kPowMulX) a2 = (uint32_t)pos[a2];
    if (top > (int32_t)kMaxPowers) return FP_E_TOO_LARGE;
    uint2 e;
    e.x = op | a1 << 2 | a2 << 17;
    e.y = (uint32_t)pos[k];
    t->ops_prog.push_back(e);
    // temporaries die after their last use (template powers stay until the walk)
    for (uint32_t o : {(w >> 2) & 0x7FFFu, w >> 17}) {
      if (op == kPowLoad || (o == (w >> 17) && op != kPowMulX)) continue;
      if (!live[o] && !tmpl[o] && last_use[o] == (int64_t)k && pos[o] >= nlive) {
        free_pos.push_back(pos[o]);
        last_use[o] = -1;  // x^(2k+1) = x^(2k) x may name one operand twice
      }
    }
  }
  t->ops_nlive = nlive;
  t->ops_nslot = nslot;
  t->ops_entries = std::max(top, nlive + nslot);

  // op records in this layout
  for (size_t i = 0; i < nops; ++i) {
    uint32_t x = t->ops[i].x;
    const int64_t j1 = (int64_t)t->ops[i].z + (t->ops[i].y & 255u);
    if ((t->ops[i].y >> 8) & 255u) t->ops[i].y = (t->ops[i].y & 0xFFFFu) | (uint32_t)pos[t->ops[i].y >> 16] << 16;
    const uint32_t S = reads[i] >= 0 ? (uint32_t)olh[reads[i]] : 0u;
    const uint32_t D = (uint32_t)olh[t->parent[j1]];
    const uint32_t pid = x >> kOpPid;
    uint32_t P;
    if (rare[pid]) {  // recomputed: z carries the base's position, m and the low bits
      const uint32_t base = redge[pid] & 0x7FFFu;
      t->ops[i].z = (redge[pid] & ~0x7FFFu) | (base == 0x7FFFu ? 0x7FFFu : (uint32_t)pos[base]);
      P = kPidRecompute;
    } else {
      P = (uint32_t)pos[pid];
    }
    x &= ~((63u << kOpS) | (63u << kOpD) | (0x7FFFu << kOpPid));
    t->ops[i].x = x | S << kOpS | D << kOpD | P << kOpPid;
  }
  t->ops_defer.clear();
  for (size_t i = 0; i < nops; ++i)
    if (t->ops[i].w >> 31) t->ops_defer.push_back(make_uint2(t->ops[i].x >> kOpPid, t->ops[i].z));
  t->ops_chain_pid.assign(N > 0 ? N - 1 : 0, 0);
  for (int64_t j = 0; j + 1 < N; ++j) {
    const int32_t p = pos[t->ctrl[j] >> kCtrlPid];
    t->ops_chain_pid[j] = p >= 0 ? (uint32_t)p : 0u;
  }
  t->ops_root_lh = root_h;
  t->ops_root_pid = t->root_pid >= 0 ? pos[t->root_pid] : -1;
  t->ops_pos_x1 = t->pid_x1 >= 0 && live[t->pid_x1] ? pos[t->pid_x1] : -1;
  t->ops_ext = 0;
  for (size_t i = 0; i < nops; ++i)
    if (((t->ops[i].y >> 8) & 255u) || (t->ops[i].x >> kOpPid) == kPidRecompute) t->ops_ext = 1;
  // template powers exist only for trees with blocks (E, B): without, their
  // positions may have been reused by temporaries, so none is reported
  for (int d = 0; d <= kMaxBlock; ++d)
    t->ops_pid_pow[d] = t->block_scheme && t->pid_pow[d] >= 0 ? pos[t->pid_pow[d]] : -1;
  return FP_OK;
}


}  // namespace

// Every index the kernels take from a schedule, checked against the array or
// table it indexes before the schedule is uploaded: a schedule that fails is
// a fault of this compiler, reported as FP_E_INTERNAL instead of sending a
// kernel outside its buffers.  Node-by-node kernel: slots 0..max_lh, powers
// [0, npow), program operands earlier in the program (dependency order).
// Grouped-op kernel: slots below nslot (positions nlive + S < entries),
// powers below entries (or rebuilt, Balanced blocks only), the coefficient
// stream read in aligned 4-element vectors within its device padding, edge
// powers of chains for nodes 0 .. nnodes - 2, and the split's marked edges.
int validate_schedule(const fp_tree* t) {
  const int64_t N = t->nnodes;
  if (N <= 0) return FP_OK;
  const int64_t npow = (int64_t)t->pow_prog.size();
  const int L = t->max_lh;
  if ((int64_t)t->ctrl.size() != N - 1 || (int64_t)t->pow_var.size() != npow ||
      (int64_t)t->pow_deg.size() != npow)
    return FP_E_INTERNAL;
  for (int64_t k = 0; k < npow; ++k) {
    const uint32_t w = t->pow_prog[k], op = w & 3u, a1 = (w >> 2) & 0x7FFFu, a2 = w >> 17;
    if (op == kPowLoad) {
      if ((int)a1 >= t->nvars) return FP_E_INTERNAL;
    } else if (op == kPowSq) {
      if ((int64_t)a1 >= k) return FP_E_INTERNAL;
    } else if (op == kPowMulX) {
      if ((int64_t)a1 >= k || (int64_t)a2 >= k) return FP_E_INTERNAL;
    } else {
      return FP_E_INTERNAL;
    }
    if (t->pow_var[k] < 0 || t->pow_var[k] >= t->nvars) return FP_E_INTERNAL;
  }
  for (int64_t j = 0; j + 1 < N; ++j) {
    const uint32_t c = t->ctrl[j];
    if ((int)((c >> kCtrlS) & 63u) > L || (int)((c >> kCtrlD) & 63u) > L || (int64_t)(c >> kCtrlPid) >= npow)
      return FP_E_INTERNAL;
  }
  if (t->root_lh < 0 || t->root_lh > L || t->root_pid >= npow) return FP_E_INTERNAL;

  const int64_t nops = (int64_t)t->ops.size(), ns = (int64_t)t->stream.size();
  const int E = t->ops_entries, nslot = t->ops_nslot;
  if (t->ops_nlive < 0 || nslot < 1 || t->ops_nlive + nslot > E) return FP_E_INTERNAL;
  if ((int64_t)t->ops_chain_pid.size() != N - 1) return FP_E_INTERNAL;
  for (const uint32_t p : t->ops_chain_pid)
    if ((int64_t)p >= E) return FP_E_INTERNAL;
  auto r4 = [](int64_t n) { return (n + kStreamAlign - 1) / kStreamAlign * kStreamAlign; };
  int64_t marked = 0;
  for (int64_t i = 0; i < nops; ++i) {
    const uint4 h = t->ops[i];
    const uint32_t kind = h.x & 3u, S = (h.x >> kOpS) & 63u, D = (h.x >> kOpD) & 63u, pid = h.x >> kOpPid;
    const int64_t len = (int64_t)(h.y & 255u) + 1, f = (h.y >> 8) & 255u, off = h.w & 0x7FFFFFFFu;
    const bool block = kind == kOpBlock || kind == kOpPartial;
    if ((int)S >= nslot || (int)D >= nslot) return FP_E_INTERNAL;
    if (pid == kPidRecompute) {  // z is the rebuild word: base | m << 15 | bits << 19
      const uint32_t base = h.z & 0x7FFFu;
      if (!t->ops_ext || !block || (base != 0x7FFFu && (int)base >= E) || t->ops_pid_pow[1] < 0)
        return FP_E_INTERNAL;
    } else {  // z is the first node; the op's nodes are non-root nodes
      if ((int)pid >= E || (int64_t)h.z + len > N - 1) return FP_E_INTERNAL;
    }
    if (kind != kOpNode) {
      if (off % kStreamAlign) return FP_E_INTERNAL;
      int64_t end = off + r4(len);
      if (f > 0) {  // a two-part run: a from off, b from the next aligned offset
        if (!t->ops_ext || !block || f >= len || (int)(h.y >> 16) >= E) return FP_E_INTERNAL;
        end = off + r4(len - f) + r4(f);
      }
      if (end > ns + kStreamAlign) return FP_E_INTERNAL;  // the device stream's padding
    }
    if (h.w >> 31) {
      if (t->ops_split <= 0 || i < t->ops_split) return FP_E_INTERNAL;
      ++marked;
    }
  }
  if (t->ops_split < 0 || (nops > 0 && t->ops_split >= nops) || marked != t->ops_ndefer ||
      (int64_t)t->ops_defer.size() != marked)
    return FP_E_INTERNAL;
  for (const uint2& e : t->ops_defer) {
    if (e.x == kPidRecompute) {
      if (!t->ops_ext || ((e.y & 0x7FFFu) != 0x7FFFu && (int)(e.y & 0x7FFFu) >= E)) return FP_E_INTERNAL;
    } else if ((int)e.x >= E) {
      return FP_E_INTERNAL;
    }
  }
  if (t->ops_root_lh < 0 || t->ops_root_lh >= nslot || t->ops_root_pid >= E) return FP_E_INTERNAL;
  for (int d = 0; d <= kMaxBlock; ++d)
    if (t->ops_pid_pow[d] >= E) return FP_E_INTERNAL;
  for (const uint2& e : t->ops_prog) {
    const uint32_t op = e.x & 3u, a1 = (e.x >> 2) & 0x7FFFu, a2 = e.x >> 17;
    if ((int64_t)e.y >= E) return FP_E_INTERNAL;
    if (op == kPowLoad) {
      if ((int)a1 >= t->nvars) return FP_E_INTERNAL;
    } else if (op == kPowSq) {
      if ((int)a1 >= E) return FP_E_INTERNAL;
    } else if (op == kPowMulX) {
      if ((int)a1 >= E || (int)a2 >= E) return FP_E_INTERNAL;
    } else {
      return FP_E_INTERNAL;
    }
  }
  return FP_OK;
}

int compile_host(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs,
                 fp_dtype coeff_type, fp_scheme scheme, const int32_t* f_table,
                 int64_t f_table_len, fp_tree* t) {
  if (nvars < 1 || nvars > FP_MAX_VARS || nterms < 0) return nvars > FP_MAX_VARS ? FP_E_TOO_LARGE : FP_E_BAD_VALUE;
  if (nterms > FP_MAX_TERMS) return FP_E_TOO_LARGE;
  if (nterms > 0 && (!exps || !coeffs)) return FP_E_BAD_VALUE;
  if (coeff_type != FP_F64 && coeff_type != FP_MODP) return FP_E_DTYPE;
  if ((int)scheme < FP_SCHEME_D || (int)scheme > FP_SCHEME_CUSTOM) return FP_E_BAD_SCHEME;
  if (scheme == FP_SCHEME_CUSTOM && (!f_table || f_table_len < 1)) return FP_E_BAD_SCHEME;
  const uint64_t P = 0xFFFFFFFF00000001ull;

  // a1: keep the non-zero terms, sort them into decreasing lex order
  std::vector<int64_t> order;
  order.reserve(nterms);
  for (int64_t i = 0; i < nterms; ++i) {
    for (int v = 0; v < nvars; ++v)
      if (exps[i * nvars + v] < 0) return FP_E_BAD_VALUE;
    if (coeff_type == FP_MODP) {
      const uint64_t c = ((const uint64_t*)coeffs)[i];
      if (c >= P) return FP_E_BAD_VALUE;
      if (c == 0) continue;
    } else {
      const double c = ((const double*)coeffs)[i];
      if (!(c == c) || c == 0.0) {
        if (c == 0.0) continue;
        return FP_E_BAD_VALUE;  // NaN coefficient
      }
    }
    order.push_back(i);
  }
  auto greater = [&](int64_t a, int64_t b) {
    for (int v = 0; v < nvars; ++v) {
      const int32_t x = exps[a * nvars + v], y = exps[b * nvars + v];
      if (x != y) return x > y;
    }
    return false;
  };
  std::stable_sort(order.begin(), order.end(), greater);
  for (size_t i = 1; i < order.size(); ++i)
    if (!greater(order[i - 1], order[i])) return FP_E_DUP_TERM;

  t->nvars = nvars;
  t->coeff_type = coeff_type;
  t->nterms_in = nterms;
  t->node_e.clear();
  t->term_of_node.clear();
  if (order.empty()) {  // the zero polynomial
    t->nnodes = 0;
    return FP_OK;
  }
  emit_with_roots(order, 0, (int64_t)order.size() - 1, 0, nvars, exps, t->node_e, t->term_of_node);
  const int64_t N = (int64_t)t->term_of_node.size();
  t->nnodes = N;
  t->parent.assign(N, -1);
  t->pd_var.assign(N, 0);
  t->pd.assign(N, 0);

  // a2: the tree, Def. 1.2 per level
  Builder bld{nvars, t->node_e, t->parent, t->pd_var, t->pd, scheme, f_table, f_table_len};
  bld.level(0, N - 1, 0);
  if (bld.status != FP_OK) return bld.status;
  t->pd_var[N - 1] = 0;
  t->pd[N - 1] = t->node_e[(N - 1) * nvars];  // root: (e_1, 0, ..., 0)

  // node coefficients
  if (coeff_type == FP_MODP) {
    t->c_u64.assign(N, 0);
    for (int64_t i = 0; i < N; ++i)
      if (t->term_of_node[i] >= 0) t->c_u64[i] = ((const uint64_t*)coeffs)[t->term_of_node[i]];
  } else {
    t->c_f64.assign(N, 0.0);
    for (int64_t i = 0; i < N; ++i)
      if (t->term_of_node[i] >= 0) t->c_f64[i] = ((const double*)coeffs)[t->term_of_node[i]];
  }

  // a3: lazy heights (children precede parents in index order)
  t->lh.assign(N, 0);
  std::vector<int32_t> lh_first(N, 0), lh_rest(N, -1);
  std::vector<uint8_t> has_child(N, 0), is_first(N, 0);
  int32_t L = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int32_t h = has_child[i] ? std::max(lh_first[i], lh_rest[i] + 1) : 0;
    t->lh[i] = h;
    L = std::max(L, h);
    const int64_t q = t->parent[i];
    if (q < 0) continue;
    if (!has_child[q]) {
      has_child[q] = 1;
      is_first[i] = 1;
      lh_first[q] = h;
    } else {
      lh_rest[q] = std::max(lh_rest[q], h);
    }
  }
  if (L > FP_MAX_LAZY_HEIGHT) return FP_E_TOO_LARGE;
  t->max_lh = L;

  // a4: distinct powers x_v^d and the program computing them:
  // x^1 = x, x^(2k) = (x^k)^2, x^(2k+1) = x^(2k) x
  std::map<std::pair<int32_t, int64_t>, int32_t> pid;
  std::vector<std::pair<int32_t, int64_t>> need;
  auto want = [&](int32_t v, int64_t d) { need.emplace_back(v, d); };
  for (int64_t i = 0; i + 1 < N; ++i) want(t->pd_var[i], t->pd[i]);
  if (t->pd[N - 1] > 0) want(0, t->pd[N - 1]);
  for (size_t k = 0; k < need.size(); ++k) {  // closure under the rule above
    const auto [v, d] = need[k];
    if (d == 1) continue;
    need.emplace_back(v, (d % 2 == 0) ? d / 2 : d - 1);
  }
  std::sort(need.begin(), need.end());
  need.erase(std::unique(need.begin(), need.end()), need.end());
  if (need.size() >= kMaxPowers) return FP_E_TOO_LARGE;
  t->pow_prog.clear();
  t->pow_var.clear();
  t->pow_deg.clear();
  for (const auto& [v, d] : need) {
    const int32_t id = (int32_t)t->pow_prog.size();
    uint32_t w;
    if (d == 1) w = kPowLoad | (uint32_t)v << 2;
    else if (d % 2 == 0) w = kPowSq | (uint32_t)pid.at({v, d / 2}) << 2;
    else w = kPowMulX | (uint32_t)pid.at({v, d - 1}) << 2 | (uint32_t)pid.at({v, 1}) << 17;
    pid[{v, d}] = id;
    t->pow_prog.push_back(w);
    t->pow_var.push_back(v);
    t->pow_deg.push_back(d);
  }

  // a5: the schedule, one control word per non-root node
  t->ctrl.assign(N - 1, 0);
  for (int64_t i = 0; i + 1 < N; ++i) {
    const int64_t q = t->parent[i];
    const uint32_t leaf = has_child[i] ? 0u : 1u;
    const uint32_t S = leaf ? 0u : (uint32_t)t->lh[i];
    t->ctrl[i] = S << kCtrlS | (uint32_t)t->lh[q] << kCtrlD | leaf << kCtrlLeaf |
                 (uint32_t)is_first[i] << kCtrlFirst |
                 (uint32_t)pid.at({t->pd_var[i], t->pd[i]}) << kCtrlPid;
  }
  // a5': group the walk into ops (fused value types).  A block is a maximal
  // subtree of at most kMaxBlock nodes (kMaxExactBlock for residues) over consecutive exponents of a
  // univariate polynomial under E or B: its shape is the scheme's own split
  // applied to a dense run, so a compile-time template evaluates it.  A
  // partial block is, for a node N with a larger subtree, N together with its
  // last children when these form a dense run of at most kMaxBlock nodes: by
  // the recursion of Def. 1.2 (p = a x^f + b, b split again by the same rule)
  // that run is the lower part b of one of the splits of N's run, so the same
  // templates evaluate it, with N's slot (c_N plus N's earlier, larger
  // children) in place of c_N.  A chain is a run j0..j1 where each node is the
  // only child of the next.
  {
    std::vector<int64_t> size(N, 1), nchild(N, 0);
    for (int64_t i = 0; i + 1 < N; ++i) {
      size[t->parent[i]] += size[i];
      nchild[t->parent[i]]++;
    }
    // blocks run over the innermost variable (the only one, for univariate
    // polynomials): its groups are univariate polynomials under the scheme
    const int bv = nvars - 1;
    const bool blocks = scheme == FP_SCHEME_E || scheme == FP_SCHEME_B;
    // residues are exact, so their kernels run a block as one loop over its
    // run (any length); the floating-point kernels use compiled templates of
    // at most kMaxBlock nodes, and a longer run (up to kMaxTwoPartBlock) as its
    // two parts under the scheme's split, joined with x^f from the table
    const bool exact_blocks = coeff_type == FP_MODP;
    const int64_t max_block = exact_blocks ? kMaxExactBlock : kMaxTwoPartBlock;
    // (blocks of 13 to 16 nodes already amortise an op: two such parts
    // measured slower, so only the Balanced scheme takes longer runs, and
    // only up to kMaxTwoPartBlock nodes, i.e. parts of at most 11)
    auto split_power_ok = [&](int64_t s) {  // a run of s nodes can form one op
      if (exact_blocks || s <= kMaxBlock) return true;
      if (scheme != FP_SCHEME_B || s > kMaxTwoPartBlock) return false;
      const int64_t f = split_count(scheme, nullptr, 0, s - 1);
      return f >= 1 && f <= kMaxBlock && s - f <= kMaxBlock && pid.count({bv, (int32_t)f}) > 0;
    };
    // nodes j0..r have consecutive exponents of x_bv and equal exponents of the others
    auto dense_run = [&](int64_t j0, int64_t r) {
      const int32_t* er = &t->node_e[r * nvars];
      for (int64_t j = j0; j < r; ++j) {
        const int32_t* ej = &t->node_e[j * nvars];
        for (int v = 0; v < bv; ++v)
          if (ej[v] != er[v]) return false;
        if (ej[bv] - er[bv] != r - j) return false;
      }
      return true;
    };
    t->block_scheme = blocks ? (int)scheme : 0;
    std::vector<int64_t> block_len(N, 0);    // at the block's first node
    std::vector<int64_t> partial_len(N, 0);  // at the partial block's first node
    std::vector<uint8_t> in_partial(N, 0);   // node lies inside a partial block
    if (blocks) {
      // qual: the subtree is a dense run of at most max_block nodes
      std::vector<uint8_t> qual(N, 0), in_block(N, 0);
      for (int64_t r = 0; r + 1 < N; ++r) {
        const int64_t s = size[r];
        qual[r] = s >= 2 && s <= max_block && r - s + 1 < (1ll << 32) && split_power_ok(s) && dense_run(r - s + 1, r);
      }
      // subtrees inside a maximal qualifying subtree (nodes in index order:
      // a subtree is the contiguous range ending at its root)
      for (int64_t r = N - 2; r >= 0; --r) {
        const int64_t q = t->parent[r];
        if (q != N - 1 && (in_block[q] || qual[q])) in_block[r] = 1;
      }
      // partial blocks: a node outside any block, with the longest suffix of
      // its children that forms a dense run with it (in a multivariate tree
      // the earlier children may be other groups); the root keeps its path
      for (int64_t r = 0; r + 1 < N; ++r) {
        if (qual[r] || in_block[r]) continue;
        int64_t s = 1, best = 1, pos = r - 1;
        while (pos >= 0 && t->parent[pos] == r && s + size[pos] <= max_block) {
          s += size[pos];
          pos -= size[pos];
          if (!dense_run(r - s + 1, r)) break;
          if (split_power_ok(s)) best = s;
        }
        s = best;
        if (s < 2) continue;
        const int64_t j0 = r - s + 1;
        if (j0 >= (1ll << 32)) continue;
        partial_len[j0] = s;
        for (int64_t j = j0; j <= r; ++j) in_partial[j] = 1;
      }
      // blocks: maximal qualifying subtrees not absorbed by a partial block
      for (int64_t r = 0; r + 1 < N; ++r)
        if (qual[r] && !in_block[r] && !in_partial[r]) block_len[r - size[r] + 1] = size[r];
    }
    auto pid_of = [&](int64_t i) { return (uint32_t)pid.at({t->pd_var[i], t->pd[i]}); };
    auto emit = [&](uint32_t kind, int64_t j0, int64_t j1) {
      const int64_t q = t->parent[j1];
      // S: the slot an op starts from (a partial block adds its last node's slot)
      const uint32_t leaf = (kind != kOpPartial && !has_child[j0]) ? 1u : 0u;
      const uint32_t S = kind == kOpPartial ? (uint32_t)t->lh[j1] : leaf ? 0u : (uint32_t)t->lh[j0];
      uint32_t x = kind | S << kOpS | (uint32_t)t->lh[q] << kOpD | leaf << kOpLeaf |
                   (uint32_t)is_first[j1] << kOpFirst | pid_of(j1) << kOpPid;
      if (kind == kOpChain) {
        bool uni = true;
        for (int64_t j = j0; j < j1; ++j) uni = uni && pid_of(j) == pid_of(j0);
        x |= (uni ? 1u : 0u) << kOpUniform;
      }
      // a floating-point block longer than kMaxBlock: the split f of its run,
      // the power x^f, and its coefficients as two aligned runs (a, then b)
      const int64_t len = j1 - j0 + 1;
      const bool two_part = (kind == kOpBlock || kind == kOpPartial) && !exact_blocks && len > kMaxBlock;
      const int64_t f = two_part ? split_count(scheme, nullptr, 0, len - 1) : 0;
      uint32_t off = 0;
      if (kind != kOpNode) {
        while (t->stream.size() % kStreamAlign) t->stream.push_back(-1);
        off = (uint32_t)t->stream.size();  // below 2^31 (FP_MAX_TERMS): w's bit 31 is a flag
        for (int64_t j = j0; j <= j1; ++j) {
          if (two_part && j == j1 - f + 1)
            while ((t->stream.size() - off) % kStreamAlign) t->stream.push_back(-1);
          t->stream.push_back(j);
        }
      }
      uint4 w;
      w.x = x;
      w.y = (uint32_t)(len - 1);
      if (two_part) w.y |= (uint32_t)f << 8 | pid.at({bv, (int32_t)f}) << 16;
      w.z = (uint32_t)j0;
      w.w = off;
      t->ops.push_back(w);
      t->op_a_node.push_back(kind == kOpNode && leaf ? j0 : -1);
      t->op_b_node.push_back(is_first[j1] ? q : -1);
    };
    t->ops.clear();
    t->op_a_node.clear();
    t->op_b_node.clear();
    t->stream.clear();
    for (int64_t i = 0; i + 1 < N;) {
      if (partial_len[i] > 0) {  // N = i + len - 1 is not a leaf: S is its slot
        const int64_t r = i + partial_len[i] - 1;
        emit(kOpPartial, i, r);
        i = r + 1;
        continue;
      }
      if (block_len[i] > 0) {
        emit(kOpBlock, i, i + block_len[i] - 1);
        i += block_len[i];
        continue;
      }
      int64_t j = i;
      while (j + 1 < N - 1 && j - i + 1 < kMaxChain && t->parent[j] == j + 1 && nchild[j + 1] == 1 &&
             block_len[j + 1] == 0)
        ++j;
      emit(j > i ? kOpChain : kOpNode, i, j);
      i = j + 1;
    }
    t->pid_x1 = pid.count({bv, 1}) ? pid.at({bv, 1}) : -1;
    for (int d = 0; d <= kMaxBlock; ++d) t->pid_pow[d] = pid.count({bv, d}) ? pid.at({bv, d}) : -1;
    if (t->pid_x1 < 0) t->block_scheme = 0;
  }

  t->root_leaf = has_child[N - 1] ? 0 : 1;
  t->root_lh = t->lh[N - 1];
  t->root_pid = t->pd[N - 1] > 0 ? pid.at({0, t->pd[N - 1]}) : -1;
  const int rc = ops_layout(t);
  return rc == FP_OK ? validate_schedule(t) : rc;
}

}  // namespace fp
