// Cholesky lambda tensor (Sec. IV.A Eq. cc12; Sec. III.A lambda tensors).
//
// V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L] is formed slab by
// slab, a slab being the blocks of V whose first-mode tile lies in a range of
// consecutive tiles (consecutive in V's packed lexicographic layout, so a slab
// is one contiguous run of V's storage).  Forming a slab is two library
// operations on the stream:
//   1. X1[p,r,q,s] = sum_L X[p,r,L] X[q,s,L]   one contraction (every block a
//      GEMM of (p,r) rows by (q,s) columns over L, both factors L-contiguous);
//   2. V[p,q,r,s]  = X1[p,r,q,s] - X1[p,s,q,r]  one pass of the pair-difference
//      kernel (the second term's planes transposed through shared memory), or
//      the two-term permuted add where a plane would not fit;
// then the contraction that reads V runs on the slab.  Both steps use the
// reading contraction's precision, so a split-precision read also forms V in
// split precision.
#include <algorithm>
#include <cstring>

#include "tamm_lambda.h"
#include "tamm_contract.h"
#include "tamm_plan.h"

namespace tamm {

namespace {

constexpr int64_t kDefaultSlabBytes = int64_t(8) << 30;

// Labels of the formation: p, q, r, s are V's modes and L the auxiliary index.
constexpr const char* kLabelX1 = "prqs";
constexpr const char* kLabelXs = "prL";
constexpr const char* kLabelX = "qsL";
constexpr const char* kLabelV = "pqrs";
const char* const kTermsV[2] = {"prqs", "psqr"};  // V(pqrs) = X1(p,r,q,s) - X1(p,s,q,r)
const double kCoefV[2] = {1.0, -1.0};

std::unique_ptr<tamm_tensor> new_tensor(tamm_ctx* ctx, int nm, const tamm_space* const* sp, int n_upper, int sym) {
  std::unique_ptr<tamm_tensor> T(new tamm_tensor());
  T->ctx = ctx;
  T->id = ctx->next_id++;
  T->nm = nm;
  T->n_upper = n_upper;
  T->sym = sym;
  for (int m = 0; m < nm; ++m) T->sp[m] = sp[m];
  return T;
}

// Some aux tile links the stored X blocks (a, b, l) and (c, d, l): their product is not identically zero.
bool linked(const tamm_tensor& X, int64_t a, int64_t b, int64_t c, int64_t d) {
  const int64_t nl = X.sp[2]->n_tiles;
  for (int64_t l = 0; l < nl; ++l) {
    const int64_t t1[3] = {a, b, l}, t2[3] = {c, d, l};
    if (X.find(t1) >= 0 && X.find(t2) >= 0) return true;
  }
  return false;
}

// Offset of the first block whose first-mode tile is >= t (n_elems if none).
int64_t first_offset(const tamm_tensor& T, int64_t t) {
  for (int64_t b = 0; b < T.n_blocks; ++b)
    if (T.tiles[(size_t)(b * T.nm)] >= t) return T.off[(size_t)b];
  return T.n_elems;
}

// The formation product has a short summed range (the aux index) over very many output tiles, so a grid of
// one CTA per tile spends much of its time on per-CTA setup and on the pipeline ramp of every tile; the
// persistent grid (one CTA per SM walking the tiles) prefetches the next tile's operands while the current
// one drains.  Measured on the O=40 V=240, 560-vector ladder: 36.1 -> 26.5 ms for the two formation GEMMs.
struct PersistentGrid {
  tamm_ctx* ctx;
  bool saved;
  explicit PersistentGrid(tamm_ctx* c) : ctx(c), saved(c->oz_persistent) { c->oz_persistent = true; }
  ~PersistentGrid() { ctx->oz_persistent = saved; }
};

void form_slab(tamm_ctx* ctx, const CholeskyLambda& lam, CholeskySlab& s, double* v_dst, int precision,
               int slices) {
  const tamm_tensor* X = lam.X;
  s.xs->data = X->data ? X->data + s.x_begin : nullptr;
  s.x1->data = lam.x1_buf;
  s.v->data = v_dst;
  {
    PersistentGrid grid(ctx);
    run_contract(ctx, 1.0, s.x1.get(), kLabelX1, 0.0, s.xs.get(), kLabelXs, X, kLabelX, precision, slices);
  }
  if (s.pair_smem)
    cuda_check(launch_cholesky_pair(ctx, v_dst, lam.x1_buf, s.d_pair_blocks, s.d_pair_items, s.n_pair_items,
                                    s.pair_smem),
               "cholesky pair kernel");
  else
    run_add(ctx, s.v.get(), kLabelV, 0.0, s.x1.get(), 2, kTermsV, kCoefV);
}

// Block and item lists of the pair-difference kernel for one slab, with every extent and offset checked
// against the block tables so that the kernel's indexing stays inside V's and X1's blocks.
void build_pair_plan(tamm_ctx* ctx, CholeskySlab& s) {
  const tamm_tensor& V = *s.v;
  const tamm_tensor& X1 = *s.x1;
  std::vector<PairBlock> blocks;
  std::vector<PairItem> items;
  size_t smem = 0;
  for (int64_t b = 0; b < V.n_blocks; ++b) {
    const int64_t* t = &V.tiles[(size_t)(b * 4)];
    const int64_t tp = t[0], tq = t[1], tr = t[2], ts = t[3];
    PairBlock pb;
    pb.np = (int32_t)V.sp[0]->size[(size_t)tp];
    pb.nq = (int32_t)V.sp[1]->size[(size_t)tq];
    pb.nr = (int32_t)V.sp[2]->size[(size_t)tr];
    pb.ns = (int32_t)V.sp[3]->size[(size_t)ts];
    const int64_t n = (int64_t)pb.np * pb.nq * pb.nr * pb.ns;
    const int64_t ta[4] = {tp, tr, tq, ts}, tb[4] = {tp, ts, tq, tr};
    const int64_t ba = X1.find(ta), bb = X1.find(tb);
    if (V.block_size(b) != n || (ba >= 0 && X1.block_size(ba) != n) || (bb >= 0 && X1.block_size(bb) != n))
      throw Error(TAMM_EINVAL, "cholesky: block extents disagree");
    pb.v_off = V.off[(size_t)b];
    pb.a_off = ba >= 0 ? X1.off[(size_t)ba] : -1;
    pb.b_off = bb >= 0 ? X1.off[(size_t)bb] : -1;
    smem = std::max(smem, (size_t)8 * (size_t)pb.ns * (size_t)(pb.nr + 1));
    const int32_t bi = (int32_t)blocks.size();
    blocks.push_back(pb);
    for (int32_t p = 0; p < pb.np; ++p) items.push_back({bi, p});
  }
  if (smem > kPairSmemMax || items.empty()) return;
  s.pair_plan.reset(new Plan(ctx));
  s.d_pair_blocks = s.pair_plan->upload(blocks);
  s.d_pair_items = s.pair_plan->upload(items);
  s.n_pair_items = (int64_t)items.size();
  s.pair_smem = smem;
}

CholeskyLambda& lambda_of(const tamm_tensor* V) {
  if (!V || !V->lambda) throw Error(TAMM_EINVAL, "cholesky: not a lambda tensor");
  return *V->lambda;
}

}  // namespace

CholeskyLambda::~CholeskyLambda() {
  if (v_buf) ctx_free(ctx, v_buf, v_bytes);
  if (x1_buf) ctx_free(ctx, x1_buf, x1_bytes);
}

std::unique_ptr<tamm_tensor> make_cholesky_tensor(tamm_ctx* ctx, const tamm_tensor* X, int64_t slab_bytes) {
  if (!X) throw Error(TAMM_EINVAL, "cholesky: null tensor");
  if (X->lambda) throw Error(TAMM_EINVAL, "cholesky: the Cholesky vectors must be a stored tensor");
  if (X->nm != 3) throw Error(TAMM_EINVAL, "cholesky: the Cholesky vectors need three modes (P, R, aux)");
  if (X->ctx != ctx) throw Error(TAMM_EINVAL, "cholesky: tensor of another context");
  if (slab_bytes < 0) throw Error(TAMM_EINVAL, "cholesky: negative slab size");
  if (slab_bytes == 0) slab_bytes = kDefaultSlabBytes;
  const tamm_space* P = X->sp[0];
  const tamm_space* R = X->sp[1];
  const tamm_space* vsp[4] = {P, P, R, R};
  const tamm_space* x1sp[4] = {P, R, P, R};
  auto V = new_tensor(ctx, 4, vsp, 2, X->sym);
  build_blocks_where(*V, [&](const int64_t* t) {
    return linked(*X, t[0], t[2], t[1], t[3]) || linked(*X, t[0], t[3], t[1], t[2]);
  });
  auto x1_all = new_tensor(ctx, 4, x1sp, -1, -1);
  build_blocks_where(*x1_all, [&](const int64_t* t) { return linked(*X, t[0], t[1], t[2], t[3]); });

  // consecutive first-mode tiles per slab while both slab buffers stay within slab_bytes
  const int64_t np = P->n_tiles;
  std::vector<int64_t> tile_bytes((size_t)np, 0);
  for (int64_t b = 0; b < V->n_blocks; ++b) tile_bytes[(size_t)V->tiles[(size_t)(b * 4)]] += 8 * V->block_size(b);
  for (int64_t b = 0; b < x1_all->n_blocks; ++b)
    tile_bytes[(size_t)x1_all->tiles[(size_t)(b * 4)]] += 8 * x1_all->block_size(b);
  std::vector<std::pair<int64_t, int64_t>> ranges;
  int64_t lo = 0, bytes = 0;
  for (int64_t t = 0; t < np; ++t) {
    if (t > lo && bytes + tile_bytes[(size_t)t] > slab_bytes) {
      ranges.push_back({lo, t});
      lo = t;
      bytes = 0;
    }
    bytes += tile_bytes[(size_t)t];
  }
  if (np > lo) ranges.push_back({lo, np});

  auto lam = std::make_shared<CholeskyLambda>();
  lam->ctx = ctx;
  lam->X = X;
  size_t vmax = 0, x1max = 0;
  for (const auto& r : ranges) {
    const int64_t t0 = r.first, t1 = r.second;
    auto in = [t0, t1](int64_t t) { return t >= t0 && t < t1; };
    CholeskySlab s;
    s.tile_lo = t0;
    s.tile_hi = t1;
    s.v = new_tensor(ctx, 4, vsp, 2, X->sym);
    build_blocks_where(*s.v, [&](const int64_t* t) { return in(t[0]) && V->find(t) >= 0; });
    if (s.v->n_blocks == 0) continue;  // nothing of V here
    s.x1 = new_tensor(ctx, 4, x1sp, -1, -1);
    build_blocks_where(*s.x1, [&](const int64_t* t) { return in(t[0]) && x1_all->find(t) >= 0; });
    s.xs = new_tensor(ctx, 3, X->sp, X->n_upper, X->sym);
    build_blocks_where(*s.xs, [&](const int64_t* t) { return in(t[0]) && X->find(t) >= 0; });
    s.v_begin = first_offset(*V, t0);
    s.x_begin = first_offset(*X, t0);
    if (!ctx->host_only) build_pair_plan(ctx, s);
    lam->form_flops += contract_flops(ctx, s.x1.get(), kLabelX1, s.xs.get(), kLabelXs, X, kLabelX);
    vmax = std::max(vmax, (size_t)s.v->n_elems * 8);
    x1max = std::max(x1max, (size_t)s.x1->n_elems * 8);
    lam->slabs.push_back(std::move(s));
  }
  lam->v_bytes = std::max<size_t>(vmax, 8);
  lam->x1_bytes = std::max<size_t>(x1max, 8);
  if (!ctx->host_only) {
    lam->v_buf = (double*)ctx_alloc(ctx, lam->v_bytes);
    lam->x1_buf = (double*)ctx_alloc(ctx, lam->x1_bytes);
  }
  V->lambda = lam;
  return V;
}

void cholesky_form(tamm_ctx* ctx, const tamm_tensor* V, tamm_tensor* out, int precision, int slices) {
  CholeskyLambda& lam = lambda_of(V);
  if (!out || out->lambda) throw Error(TAMM_EINVAL, "cholesky form: the output must be a stored tensor");
  if (lam.ctx != ctx || out->ctx != ctx) throw Error(TAMM_EINVAL, "cholesky form: tensor of another context");
  if (ctx->group_active) throw Error(TAMM_EUNSUPPORTED, "cholesky form cannot be issued inside a contraction group");
  bool same = out->nm == 4 && out->n_blocks == V->n_blocks && out->tiles == V->tiles;
  for (int m = 0; same && m < 4; ++m) same = out->sp[m] == V->sp[m];
  if (!same) throw Error(TAMM_EINVAL, "cholesky form: the output's spaces or block table differ from V's");
  require_device(ctx);
  if (out->n_elems && !out->data) throw Error(TAMM_EINVAL, "cholesky form: output has no device storage");
  if (out->data && out->data == lam.X->data) throw Error(TAMM_EINVAL, "cholesky form: output aliases X");
  for (auto& s : lam.slabs) form_slab(ctx, lam, s, out->data + s.v_begin, precision, slices);
}

void run_contract_lambda(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                         const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb, int precision,
                         int slices) {
  if (A->lambda && B->lambda) throw Error(TAMM_EUNSUPPORTED, "contract: both operands are lambda tensors");
  const tamm_tensor* Lt = A->lambda ? A : B;
  CholeskyLambda& lam = *Lt->lambda;
  if (lam.ctx != ctx) throw Error(TAMM_EINVAL, "contract: lambda tensor of another context");
  if (ctx->group_active)
    throw Error(TAMM_EUNSUPPORTED, "contract: a lambda tensor cannot be read inside a contraction group");
  if (!C) throw Error(TAMM_EINVAL, "contract: null tensor");
  if (C->data && C->data == lam.X->data) throw Error(TAMM_EINVAL, "contract: output aliases the Cholesky vectors");
  require_device(ctx);
  bool first = true;
  for (auto& slab : lam.slabs) {
    form_slab(ctx, lam, slab, lam.v_buf, precision, slices);
    run_contract(ctx, alpha, C, lc, first ? beta : 1.0, A->lambda ? slab.v.get() : A, la,
                 B->lambda ? slab.v.get() : B, lb, precision, slices);
    first = false;
  }
  if (first) {
    // V stores no block: the product is zero and C = beta * C
    ContractLayout lay(ctx, C, lc, A, la, B, lb);
    if (C->lambda) throw Error(TAMM_EUNSUPPORTED, "contract: a lambda tensor is read-only");
    if (beta != 0.0 && beta != 1.0) throw Error(TAMM_EINVAL, "contract: beta must be 0 (=) or 1 (+=)");
    if (C->n_elems && !C->data) throw Error(TAMM_EINVAL, "contract: output has no device storage");
    if (beta == 0.0 && C->n_elems)
      cuda_check(cudaMemsetAsync(C->data, 0, (size_t)C->n_elems * 8, ctx->stream), "memset");
  }
}

}  // namespace tamm
