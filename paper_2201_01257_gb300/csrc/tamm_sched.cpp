// Scheduler: deferred execution of recorded operations by dependency level
// (Sec. III.A: operations are declared and run through a scheduler; Sec.
// III.B: a data-flow analysis marks two operations as conflicting when they
// share a tensor and one of them updates it, and a levelized execution runs
// each batch of mutually independent operations together).  Host logic only:
// every operation runs through the same entry points as a direct call, and
// the split-precision contractions of a level run as one contraction group.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tamm_lambda.h"
#include "tamm_plan.h"

using namespace tamm;

namespace {

enum OpKind { kContract, kAdd, kEnergy };

struct SchedOp {
  OpKind kind;
  double alpha = 0.0, beta = 0.0;
  tamm_tensor* c = nullptr;
  const tamm_tensor* a = nullptr;
  const tamm_tensor* b = nullptr;
  std::string lc, la, lb;
  int precision = 0, slices = 0;
  std::vector<std::string> terms;  // add: source label orders
  std::vector<double> coef;        // add: their factors
  double* result = nullptr;        // energy: device result
};

// A storage range: device bytes, or (no storage) the tensor object itself.
struct Range {
  const void* p;
  size_t n;
};

bool overlap(const Range& x, const Range& y) {
  const char* a = (const char*)x.p;
  const char* b = (const char*)y.p;
  return a < b + y.n && b < a + x.n;
}

Range storage(const tamm_tensor* t) {
  if (t->data && t->n_elems) return {t->data, (size_t)t->n_elems * 8};
  return {t, 1};
}

void reads_of(const tamm_tensor* t, std::vector<Range>& out) {
  if (t->lambda) {
    out.push_back({t, 1});
    out.push_back(storage(t->lambda->X));
  } else {
    out.push_back(storage(t));
  }
}

void access(const SchedOp& op, std::vector<Range>& reads, std::vector<Range>& writes) {
  reads.clear();
  writes.clear();
  switch (op.kind) {
    case kContract:
      reads_of(op.a, reads);
      reads_of(op.b, reads);
      if (op.beta != 0.0) reads.push_back(storage(op.c));
      writes.push_back(storage(op.c));
      break;
    case kAdd:
      reads_of(op.a, reads);
      if (op.beta != 0.0) reads.push_back(storage(op.c));
      writes.push_back(storage(op.c));
      break;
    case kEnergy:
      reads_of(op.a, reads);
      reads_of(op.b, reads);
      writes.push_back({op.result, 8});
      break;
  }
}

bool any_overlap(const std::vector<Range>& x, const std::vector<Range>& y) {
  for (const auto& u : x)
    for (const auto& v : y)
      if (overlap(u, v)) return true;
  return false;
}

bool is_split(int precision) { return precision == TAMM_PREC_OZAKI_BF16 || precision == TAMM_PREC_BF16X3; }

template <class F>
tamm_status sched_guard(tamm_ctx* ctx, F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return TAMM_ENOMEM;
  }
}

void check_labels(const tamm_tensor* t, const char* l, const char* what) {
  if (!t || !l) throw Error(TAMM_EINVAL, "%s: null argument", what);
  if ((int)strlen(l) != t->nm) throw Error(TAMM_EINVAL, "%s: label string must have one label per mode", what);
}

}  // namespace

struct tamm_sched {
  tamm_ctx* ctx = nullptr;
  std::vector<SchedOp> ops;

  // level of every operation: one more than the highest earlier conflicting operation's level
  std::vector<int> levels() const {
    std::vector<int> lev(ops.size(), 0);
    std::vector<std::vector<Range>> r(ops.size()), w(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) access(ops[i], r[i], w[i]);
    for (size_t i = 0; i < ops.size(); ++i)
      for (size_t j = 0; j < i; ++j)
        if (any_overlap(w[j], r[i]) || any_overlap(w[j], w[i]) || any_overlap(r[j], w[i]))
          lev[i] = std::max(lev[i], lev[j] + 1);
    return lev;
  }
};

extern "C" tamm_status tamm_sched_create(tamm_ctx* ctx, tamm_sched** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return sched_guard(ctx, [&] {
    tamm_sched* s = new tamm_sched();
    s->ctx = ctx;
    *out = s;
    return TAMM_OK;
  });
}

extern "C" void tamm_sched_destroy(tamm_sched* s) { delete s; }

extern "C" tamm_status tamm_sched_contract(tamm_sched* s, double alpha, tamm_tensor* C, const char* lc, double beta,
                                           const tamm_tensor* A, const char* la, const tamm_tensor* B,
                                           const char* lb, int precision, int slices) {
  if (!s) return TAMM_EINVAL;
  return sched_guard(s->ctx, [&] {
    check_labels(C, lc, "sched contract");
    check_labels(A, la, "sched contract");
    check_labels(B, lb, "sched contract");
    SchedOp op;
    op.kind = kContract;
    op.alpha = alpha;
    op.beta = beta;
    op.c = C;
    op.a = A;
    op.b = B;
    op.lc = lc;
    op.la = la;
    op.lb = lb;
    op.precision = precision;
    op.slices = slices;
    s->ops.push_back(std::move(op));
    return TAMM_OK;
  });
}

extern "C" tamm_status tamm_sched_add(tamm_sched* s, tamm_tensor* C, const char* lc, double beta,
                                      const tamm_tensor* A, int n_terms, const char* const* la, const double* alpha) {
  if (!s) return TAMM_EINVAL;
  return sched_guard(s->ctx, [&] {
    check_labels(C, lc, "sched add");
    if (n_terms < 1 || n_terms > kMaxAddTerms || !la || !alpha)
      throw Error(TAMM_EINVAL, "sched add: 1..%d terms", kMaxAddTerms);
    SchedOp op;
    op.kind = kAdd;
    op.beta = beta;
    op.c = C;
    op.a = A;
    op.lc = lc;
    for (int t = 0; t < n_terms; ++t) {
      check_labels(A, la[t], "sched add");
      op.terms.push_back(la[t]);
      op.coef.push_back(alpha[t]);
    }
    s->ops.push_back(std::move(op));
    return TAMM_OK;
  });
}

extern "C" tamm_status tamm_sched_energy(tamm_sched* s, double alpha, const tamm_tensor* A, const char* la,
                                         const tamm_tensor* B, const char* lb, double* result_device) {
  if (!s) return TAMM_EINVAL;
  return sched_guard(s->ctx, [&] {
    check_labels(A, la, "sched energy");
    check_labels(B, lb, "sched energy");
    if (!result_device) throw Error(TAMM_EINVAL, "sched energy: null result pointer");
    SchedOp op;
    op.kind = kEnergy;
    op.alpha = alpha;
    op.a = A;
    op.b = B;
    op.la = la;
    op.lb = lb;
    op.result = result_device;
    s->ops.push_back(std::move(op));
    return TAMM_OK;
  });
}

extern "C" tamm_status tamm_sched_levels(tamm_sched* s, int* n_ops, int* n_levels, int* op_level) {
  if (!s) return TAMM_EINVAL;
  return sched_guard(s->ctx, [&] {
    const std::vector<int> lev = s->levels();
    if (n_ops) *n_ops = (int)lev.size();
    if (n_levels) *n_levels = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end()) + 1;
    if (op_level && !lev.empty()) memcpy(op_level, lev.data(), lev.size() * sizeof(int));
    return TAMM_OK;
  });
}

extern "C" tamm_status tamm_sched_execute(tamm_sched* s) {
  if (!s) return TAMM_EINVAL;
  tamm_ctx* ctx = s->ctx;
  return sched_guard(ctx, [&]() -> tamm_status {
    if (ctx->group_active) throw Error(TAMM_EINVAL, "sched execute: a contraction group is open");
    const std::vector<int> lev = s->levels();
    const int n_levels = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end()) + 1;
    auto run_contract_op = [&](const SchedOp& op) {
      return tamm_contract(ctx, op.alpha, op.c, op.lc.c_str(), op.beta, op.a, op.la.c_str(), op.b, op.lb.c_str(),
                           op.precision, op.slices);
    };
    for (int L = 0; L < n_levels; ++L) {
      std::vector<const SchedOp*> grouped, single, adds, energies;
      for (size_t i = 0; i < s->ops.size(); ++i) {
        if (lev[i] != L) continue;
        const SchedOp& op = s->ops[i];
        if (op.kind == kAdd) adds.push_back(&op);
        else if (op.kind == kEnergy) energies.push_back(&op);
        else if (is_split(op.precision) && !op.a->lambda && !op.b->lambda) grouped.push_back(&op);
        else single.push_back(&op);
      }
      if (!grouped.empty()) {
        tamm_status st = tamm_group_begin(ctx);
        if (st != TAMM_OK) return st;
        for (const SchedOp* op : grouped) {
          st = run_contract_op(*op);
          if (st != TAMM_OK) {
            const std::string msg = ctx->last_error;
            tamm_group_cancel(ctx);
            ctx->last_error = msg;
            return st;
          }
        }
        st = tamm_group_end(ctx);
        if (st != TAMM_OK) return st;
      }
      for (const SchedOp* op : single) {
        const tamm_status st = run_contract_op(*op);
        if (st != TAMM_OK) return st;
      }
      for (const SchedOp* op : adds) {
        std::vector<const char*> la;
        for (const auto& t : op->terms) la.push_back(t.c_str());
        const tamm_status st = tamm_add(ctx, op->c, op->lc.c_str(), op->beta, op->a, (int)la.size(), la.data(),
                                        op->coef.data());
        if (st != TAMM_OK) return st;
      }
      for (const SchedOp* op : energies) {
        const tamm_status st = tamm_energy_async(ctx, op->alpha, op->a, op->la.c_str(), op->b, op->lb.c_str(),
                                                 op->result);
        if (st != TAMM_OK) return st;
      }
    }
    ctx->last_error.clear();
    return TAMM_OK;
  });
}
