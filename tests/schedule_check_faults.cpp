// Planted faults for the compiler's schedule check (validate_schedule): each
// case copies a compiled tree, corrupts one index that the kernels take from
// its schedule, and expects FP_E_INTERNAL; every tree as compiled passes.
// Host only; built with g++ and run by tests/test_schedule_check.py.
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "tree.hpp"

namespace {

int failures = 0;

void expect(const char* what, int got, int want) {
  std::printf("%-44s %s\n", what, got == want ? "ok" : "MISSED");
  if (got != want) ++failures;
}

fp_tree compile(int nvars, const std::vector<int32_t>& exps, fp_scheme scheme, bool modp) {
  const int64_t n = (int64_t)exps.size() / nvars;
  std::vector<double> cf(n);
  std::vector<uint64_t> cu(n);
  for (int64_t i = 0; i < n; ++i) {
    cf[i] = 1.0 + (double)(i % 7) / 8.0;
    cu[i] = 3 + (uint64_t)i;
  }
  fp_tree t;
  const int rc = fp::compile_host(nvars, n, exps.data(), modp ? (const void*)cu.data() : (const void*)cf.data(),
                                  modp ? FP_MODP : FP_F64, scheme, nullptr, 0, &t);
  if (rc != FP_OK) {
    std::printf("compile failed: %d\n", rc);
    ++failures;
  }
  return t;
}

std::vector<int32_t> dense(int64_t k) {
  std::vector<int32_t> e(k);
  for (int64_t i = 0; i < k; ++i) e[i] = (int32_t)(k - 1 - i);
  return e;
}

std::vector<int32_t> graded2(int deg) {  // all (a, b) with a + b <= deg, decreasing lex
  std::vector<int32_t> e;
  for (int a = deg; a >= 0; --a)
    for (int b = deg - a; b >= 0; --b) {
      e.push_back(a);
      e.push_back(b);
    }
  return e;
}

int64_t r4(int64_t n) { return (n + fp::kStreamAlign - 1) / fp::kStreamAlign * fp::kStreamAlign; }

// first op satisfying pred, or -1
int64_t find(const fp_tree& t, const std::function<bool(const uint4&)>& pred) {
  for (size_t i = 0; i < t.ops.size(); ++i)
    if (pred(t.ops[i])) return (int64_t)i;
  return -1;
}

uint32_t kind(const uint4& h) { return h.x & 3u; }
uint32_t pid(const uint4& h) { return h.x >> fp::kOpPid; }
uint32_t f_of(const uint4& h) { return (h.y >> 8) & 255u; }
int64_t len(const uint4& h) { return (int64_t)(h.y & 255u) + 1; }

void fault(const char* what, const fp_tree& base, const std::function<bool(fp_tree&)>& corrupt) {
  fp_tree t = base;
  if (!corrupt(t)) {
    std::printf("%-44s NOT APPLICABLE\n", what);
    ++failures;
    return;
  }
  expect(what, fp::validate_schedule(&t), FP_E_INTERNAL);
}

}  // namespace

int main() {
  using namespace fp;
  // a 10007-term Balanced tree: two-part blocks, rebuilt powers, the split
  const fp_tree bal = compile(1, dense(10007), FP_SCHEME_B, false);
  // a bivariate Estrin tree: partial blocks, groups of the outer variable
  const fp_tree biv = compile(2, graded2(30), FP_SCHEME_E, false);
  // a mod-p Balanced tree: blocks of up to 64 nodes
  const fp_tree mod = compile(1, dense(3000), FP_SCHEME_B, true);
  // a Horner tree: chains
  const fp_tree hor = compile(1, dense(200), FP_SCHEME_H, false);
  expect("Balanced 10007 as compiled", validate_schedule(&bal), FP_OK);
  expect("bivariate Estrin as compiled", validate_schedule(&biv), FP_OK);
  expect("mod-p Balanced 3000 as compiled", validate_schedule(&mod), FP_OK);
  expect("Horner 200 as compiled", validate_schedule(&hor), FP_OK);

  const auto is_block = [](const uint4& h) { return kind(h) == kOpBlock || kind(h) == kOpPartial; };
  const auto plain = [&](const uint4& h) { return pid(h) != kPidRecompute; };

  // node-by-node schedule
  fault("ctrl: slot above the lazy height", bal, [](fp_tree& t) {
    t.ctrl[0] = (t.ctrl[0] & ~(63u << kCtrlS)) | (uint32_t)(t.max_lh + 1) << kCtrlS;
    return t.max_lh + 1 < 64;
  });
  fault("ctrl: power beyond the program", bal, [](fp_tree& t) {
    t.ctrl[0] = (t.ctrl[0] & ((1u << kCtrlPid) - 1)) | (uint32_t)t.pow_prog.size() << kCtrlPid;
    return true;
  });
  fault("program: square of a later power", bal, [](fp_tree& t) {
    for (size_t k = 0; k < t.pow_prog.size(); ++k)
      if ((t.pow_prog[k] & 3u) == kPowSq) {
        t.pow_prog[k] = kPowSq | (uint32_t)k << 2;
        return true;
      }
    return false;
  });
  fault("program: load of a missing variable", biv, [](fp_tree& t) {
    t.pow_prog[0] = kPowLoad | (uint32_t)t.nvars << 2;
    return (t.pow_prog.size() > 0);
  });
  fault("root power beyond the program", bal, [](fp_tree& t) {
    t.root_pid = (int)t.pow_prog.size();
    return true;
  });

  // grouped schedule: op records
  fault("op: slot read beyond the table", biv, [](fp_tree& t) {
    t.ops[0].x = (t.ops[0].x & ~(63u << kOpS)) | (uint32_t)t.ops_nslot << kOpS;
    return t.ops_nslot < 64;
  });
  fault("op: parent slot beyond the table", bal, [](fp_tree& t) {
    t.ops[0].x = (t.ops[0].x & ~(63u << kOpD)) | (uint32_t)t.ops_nslot << kOpD;
    return t.ops_nslot < 64;
  });
  fault("op: edge power beyond the table", bal, [&](fp_tree& t) {
    const int64_t i = find(t, plain);
    if (i < 0) return false;
    t.ops[i].x = (t.ops[i].x & ((1u << kOpPid) - 1)) | (uint32_t)t.ops_entries << kOpPid;
    return t.ops_entries < (int)kPidRecompute;
  });
  fault("op: rebuilt power outside the extended kernel", bal, [&](fp_tree& t) {
    t.ops_ext = 0;
    return find(t, [](const uint4& h) { return pid(h) == kPidRecompute; }) >= 0;
  });
  fault("op: rebuilt power from a base beyond the table", bal, [&](fp_tree& t) {
    const int64_t i = find(t, [](const uint4& h) { return pid(h) == kPidRecompute; });
    if (i < 0) return false;
    t.ops[i].z = (t.ops[i].z & ~0x7FFFu) | (uint32_t)t.ops_entries;
    return true;
  });
  fault("op: rebuilt power on a chain", hor, [&](fp_tree& t) {
    const int64_t i = find(t, [](const uint4& h) { return kind(h) == kOpChain; });
    if (i < 0) return false;
    t.ops_ext = 1;
    t.ops[i].x |= kPidRecompute << kOpPid;
    return true;
  });
  fault("op: nodes past the last non-root node", biv, [&](fp_tree& t) {
    const int64_t i = find(t, plain);
    if (i < 0) return false;
    t.ops[i].z = (uint32_t)(t.nnodes - 1);
    return true;
  });
  fault("op: stream offset not aligned", bal, [&](fp_tree& t) {
    const int64_t i = find(t, is_block);
    if (i < 0) return false;
    t.ops[i].w += 1;
    return true;
  });
  fault("op: stream run past the padding", bal, [&](fp_tree& t) {
    const int64_t i = find(t, [&](const uint4& h) { return is_block(h) && len(h) >= 5; });
    if (i < 0) return false;
    t.ops[i].w = (t.ops[i].w & 0x80000000u) | (uint32_t)r4((int64_t)t.stream.size());
    return true;
  });
  fault("op: mod-p run past the padding", mod, [&](fp_tree& t) {
    const int64_t i = find(t, [&](const uint4& h) { return is_block(h) && len(h) > 16; });
    if (i < 0) return false;
    t.ops[i].w = (t.ops[i].w & 0x80000000u) | (uint32_t)r4((int64_t)t.stream.size() - len(t.ops[i]) + 8);
    return true;
  });
  fault("op: two-part split not below the length", bal, [&](fp_tree& t) {
    const int64_t i = find(t, [](const uint4& h) { return f_of(h) > 0; });
    if (i < 0) return false;
    t.ops[i].y = (t.ops[i].y & ~(255u << 8)) | (uint32_t)len(t.ops[i]) << 8;
    return true;
  });
  fault("op: two-part x^f beyond the table", bal, [&](fp_tree& t) {
    const int64_t i = find(t, [](const uint4& h) { return f_of(h) > 0; });
    if (i < 0) return false;
    t.ops[i].y = (t.ops[i].y & 0xFFFFu) | (uint32_t)t.ops_entries << 16;
    return true;
  });
  fault("op: two-part run outside the extended kernel", bal, [&](fp_tree& t) {
    t.ops_ext = 0;
    return find(t, [](const uint4& h) { return f_of(h) > 0; }) >= 0;
  });

  // the split
  fault("split: root edge marked before the split", bal, [&](fp_tree& t) {
    if (t.ops_split <= 0) return false;
    t.ops[0].w |= 0x80000000u;
    ++t.ops_ndefer;
    t.ops_defer.push_back(t.ops_defer.empty() ? make_uint2(0, 0) : t.ops_defer[0]);
    return true;
  });
  fault("split: deferred-edge count", bal, [&](fp_tree& t) {
    ++t.ops_ndefer;
    return t.ops_split > 0;
  });
  fault("split: deferred edge power beyond the table", bal, [&](fp_tree& t) {
    if (t.ops_defer.empty()) return false;
    t.ops_defer[0].x = (uint32_t)t.ops_entries;
    return true;
  });
  fault("split: first op beyond the list", bal, [&](fp_tree& t) {
    t.ops_split = (int64_t)t.ops.size();
    return true;
  });

  // table layout and the program of the grouped kernel
  fault("layout: root slot beyond the table", bal, [](fp_tree& t) {
    t.ops_root_lh = t.ops_nslot;
    return true;
  });
  fault("layout: root power beyond the table", bal, [](fp_tree& t) {
    t.ops_root_pid = t.ops_entries;
    return true;
  });
  fault("layout: template power beyond the table", bal, [](fp_tree& t) {
    t.ops_pid_pow[2] = t.ops_entries;
    return true;
  });
  fault("layout: slots past the entries", bal, [](fp_tree& t) {
    t.ops_entries = t.ops_nlive + t.ops_nslot - 1;
    return true;
  });
  fault("layout: chain edge power beyond the table", biv, [](fp_tree& t) {
    if (t.ops_chain_pid.empty()) return false;
    t.ops_chain_pid.back() = (uint32_t)t.ops_entries;
    return true;
  });
  fault("program (grouped): destination beyond the table", bal, [](fp_tree& t) {
    if (t.ops_prog.empty()) return false;
    t.ops_prog.back().y = (uint32_t)t.ops_entries;
    return true;
  });
  fault("program (grouped): load of a missing variable", biv, [](fp_tree& t) {
    if (t.ops_prog.empty()) return false;
    t.ops_prog[0].x = kPowLoad | (uint32_t)t.nvars << 2;
    return true;
  });
  std::printf("failures: %d\n", failures);
  return failures;
}
