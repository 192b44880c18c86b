// Host planner.  For C(lc) = beta*C + alpha*A(la)*B(lb) it decides which
// operand is the GEMM's left side, which operand/output blocks need an index
// permutation to reach (free | summed) x (summed | free) matrix order, and
// enumerates every nonzero block pair grouped by output block (the paper's
// "series of matrix multiplications and transpositions" over non-zero blocks,
// Sec. I and Sec. III.B).  Plans are cached per context.
#include <algorithm>
#include <cstring>

#include "tamm_plan.h"
#include "tamm_contract.h"
#include "tamm_lambda.h"

namespace tamm {

// ------------------------------------------------------------- label sets

void Labels::add(const tamm_tensor* T, const char* l, int which, const char* what) {
  if (!T) throw Error(TAMM_EINVAL, "%s: null tensor", what);
  if (!l || (int)strlen(l) != T->nm) throw Error(TAMM_EINVAL, "%s: label string must have one label per mode", what);
  for (int m = 0; m < T->nm; ++m) {
    int id = -1;
    for (int i = 0; i < n; ++i)
      if (name[i] == l[m]) id = i;
    if (id < 0) {
      if (n >= kMaxLabels) throw Error(TAMM_EINVAL, "%s: too many labels", what);
      id = n++;
      name[id] = l[m];
      sp[id] = nullptr;
      for (int w = 0; w < 3; ++w) pos[w][id] = -1;
    }
    if (pos[which][id] >= 0) throw Error(TAMM_EINVAL, "%s: label '%c' repeated in one tensor", what, l[m]);
    pos[which][id] = m;
    if (sp[id] && sp[id] != T->sp[m])
      throw Error(TAMM_EINVAL, "%s: label '%c' bound to two different index spaces", what, l[m]);
    sp[id] = T->sp[m];
  }
}

int Labels::find(char c) const {
  for (int i = 0; i < n; ++i)
    if (name[i] == c) return i;
  return -1;
}

static void require_data(const tamm_tensor* T, const char* what) {
  if (T->lambda) throw Error(TAMM_EUNSUPPORTED, "%s: a lambda tensor only feeds contractions as an input", what);
  if (T->n_elems && !T->data) throw Error(TAMM_EINVAL, "%s: tensor has no device storage (bind or allocate)", what);
}

// ---------------------------------------------------------- permuted adds

// Per destination block, the source block and strides for each term.
std::vector<AddBlock> build_add_blocks(const tamm_tensor& D, const char* ld, const tamm_tensor& S, int n_terms,
                                       const char* const* ls) {
  if (D.nm > kMaxKernelModes) throw Error(TAMM_EUNSUPPORTED, "add: at most %d modes", kMaxKernelModes);
  int posS[kMaxAddTerms][kMaxModes];  // for each term, S mode holding D mode m's label
  for (int t = 0; t < n_terms; ++t) {
    for (int m = 0; m < D.nm; ++m) {
      const char* p = strchr(ls[t], ld[m]);
      posS[t][m] = (int)(p - ls[t]);
    }
  }
  std::vector<AddBlock> out((size_t)D.n_blocks);
  for (int64_t b = 0; b < D.n_blocks; ++b) {
    AddBlock& ab = out[(size_t)b];
    memset(&ab, 0, sizeof(ab));
    const int64_t* dt = &D.tiles[(size_t)(b * D.nm)];
    ab.dst_off = D.off[(size_t)b];
    ab.n = D.block_size(b);
    if (ab.n >= (int64_t(1) << 31)) throw Error(TAMM_EUNSUPPORTED, "add: a block of 2^31 or more elements");
    ab.nm = D.nm;
    for (int m = 0; m < D.nm; ++m) ab.dim[m] = (int32_t)D.sp[m]->size[(size_t)dt[m]];
    for (int t = 0; t < kMaxAddTerms; ++t) ab.src_off[t] = -1;
    for (int t = 0; t < n_terms; ++t) {
      int64_t st[kMaxModes];
      for (int m = 0; m < D.nm; ++m) st[posS[t][m]] = dt[m];
      const int64_t sb = S.find(st);
      if (sb < 0) continue;
      int64_t stride[kMaxModes], s = 1;
      for (int q = S.nm - 1; q >= 0; --q) {
        stride[q] = s;
        s *= S.sp[q]->size[(size_t)st[q]];
      }
      ab.src_off[t] = S.off[(size_t)sb];
      for (int m = 0; m < D.nm; ++m) ab.sstride[t][m] = (int32_t)stride[posS[t][m]];
    }
    // transposition: the terms that read the last destination mode with a stride must all read one
    // other destination mode contiguously, which then becomes the tile's row mode
    ab.tmode = -1;
    bool ok = D.nm >= 2 && ab.dim[D.nm - 1] > 1;
    int tm = -1;
    for (int t = 0; t < n_terms && ok; ++t) {
      if (ab.src_off[t] < 0 || ab.sstride[t][D.nm - 1] == 1) continue;
      int p = -1;
      for (int m = 0; m < D.nm - 1; ++m)
        if (ab.sstride[t][m] == 1 && ab.dim[m] > 1) p = m;
      if (p < 0 || (tm >= 0 && p != tm)) ok = false;
      tm = p;
    }
    if (ok && tm >= 0) ab.tmode = tm;
  }
  return out;
}

std::vector<ChunkItem> build_chunks(const std::vector<AddBlock>& blocks) {
  std::vector<ChunkItem> items;
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int64_t s = 0; s < blocks[b].n; s += kChunk) items.push_back({(int32_t)b, 0, s});
  return items;
}

// Tiles of the blocks that take the transposition path; the other blocks get chunks.
static void build_add_items(const std::vector<AddBlock>& blocks, std::vector<ChunkItem>& chunks,
                            std::vector<TileItem>& tiles) {
  for (size_t b = 0; b < blocks.size(); ++b) {
    const AddBlock& B = blocks[b];
    if (B.tmode < 0) {
      for (int64_t s = 0; s < B.n; s += kChunk) chunks.push_back({(int32_t)b, 0, s});
      continue;
    }
    const int p = B.tmode, q = B.nm - 1;
    int n_trans = 0;
    for (int t = 0; t < kMaxAddTerms; ++t)
      if (B.src_off[t] >= 0 && B.sstride[t][q] != 1) ++n_trans;
    int64_t outer = 1;
    for (int m = 0; m < B.nm; ++m)
      if (m != p && m != q) outer *= B.dim[m];
    for (int32_t p0 = 0; p0 < B.dim[p]; p0 += kAddTile)
      for (int32_t q0 = 0; q0 < B.dim[q]; q0 += kAddTile) {
        const int64_t tp = std::min<int64_t>(kAddTile, B.dim[p] - p0), tq = std::min<int64_t>(kAddTile, B.dim[q] - q0);
        // about 4096 elements per item, as many planes as the staging buffer holds
        int64_t per = std::max<int64_t>(1, 4096 / (tp * tq));
        per = std::min<int64_t>(per, kAddMaxOuter);
        if (n_trans) per = std::max<int64_t>(1, std::min<int64_t>(per, kAddTileSmem / (n_trans * tp * (tq + 1))));
        for (int64_t o = 0; o < outer; o += per)
          tiles.push_back({(int32_t)b, p0, q0, (int32_t)o, (int32_t)std::min<int64_t>(per, outer - o), 0});
      }
  }
}

AddPlan::AddPlan(tamm_ctx* c, const tamm_tensor& D, const char* ld, const tamm_tensor& S, int terms,
                 const char* const* ls)
    : Plan(c), n_terms(terms) {
  auto blocks = build_add_blocks(D, ld, S, terms, ls);
  std::vector<ChunkItem> items;
  std::vector<TileItem> tiles;
  build_add_items(blocks, items, tiles);
  n_items = (int64_t)items.size();
  n_tiles = (int64_t)tiles.size();
  nm = D.nm;
  if (n_tiles) d_tiles = upload(tiles);
  d_blocks = upload(blocks);
  d_items = upload(items);
}

void AddPlan::run(double* dst, const double* src, double beta, const double* alpha,
                  const double* scale_device) const {
  cuda_check(launch_add(ctx, dst, src, d_blocks, d_items, n_items, n_terms, beta, alpha, scale_device, nm, d_tiles,
                        n_tiles),
             "add kernel");
}

template <class P, class... Args>
static P* cached(tamm_ctx* ctx, const std::string& key, Args&&... args) {
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) return static_cast<P*>(it->second.get());
  P* p = new P(ctx, std::forward<Args>(args)...);
  ctx->plans[key].reset(p);
  return p;
}

static std::string tid(const tamm_tensor* T) { return std::to_string(T->id); }

void run_add(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A, int n_terms,
             const char* const* la, const double* alpha, const double* scale_device) {
  if (!C || !A || !lc || !la || !alpha) throw Error(TAMM_EINVAL, "add: null argument");
  if (n_terms < 1 || n_terms > kMaxAddTerms) throw Error(TAMM_EINVAL, "add: 1..%d terms", kMaxAddTerms);
  if (beta != 0.0 && beta != 1.0) throw Error(TAMM_EINVAL, "add: beta must be 0 or 1");
  if (C == A || (C->data && C->data == A->data)) throw Error(TAMM_EINVAL, "add: output aliases the input");
  std::string key = "add|" + tid(C) + "|" + lc + "|" + tid(A);
  for (int t = 0; t < n_terms; ++t) {
    Labels L;
    L.add(C, lc, 0, "add");
    L.add(A, la[t], 1, "add");
    for (int i = 0; i < L.n; ++i)
      if ((L.pos[0][i] >= 0) != (L.pos[1][i] >= 0))
        throw Error(TAMM_EINVAL, "add: label '%c' must appear in both tensors", L.name[i]);
    key += std::string("|") + la[t];
  }
  require_data(C, "add");
  require_data(A, "add");
  AddPlan* p = cached<AddPlan>(ctx, key, *C, lc, *A, n_terms, la);
  p->run(C->data, A->data, beta, alpha, scale_device);
}

// -------------------------------------------------------------- reductions

struct EnergyPlan : Plan {
  AddBlock* d_blocks = nullptr;
  ChunkItem* d_items = nullptr;
  int64_t n_items = 0;
  EnergyPlan(tamm_ctx* c, const tamm_tensor& A, const char* la, const tamm_tensor& B, const char* lb) : Plan(c) {
    const char* ls[1] = {lb};
    auto blocks = build_add_blocks(A, la, B, 1, ls);
    auto items = build_chunks(blocks);
    n_items = (int64_t)items.size();
    d_blocks = upload(blocks);
    d_items = upload(items);
  }
};

void run_energy(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la, const tamm_tensor* B,
                const char* lb, double* out_device) {
  Labels L;
  L.add(A, la, 1, "energy");
  L.add(B, lb, 2, "energy");
  for (int i = 0; i < L.n; ++i)
    if ((L.pos[1][i] >= 0) != (L.pos[2][i] >= 0))
      throw Error(TAMM_EINVAL, "energy: label '%c' must appear in both tensors", L.name[i]);
  require_data(A, "energy");
  require_data(B, "energy");
  std::string key = "energy|" + tid(A) + "|" + la + "|" + tid(B) + "|" + lb;
  EnergyPlan* p = cached<EnergyPlan>(ctx, key, *A, la, *B, lb);
  const int64_t n = std::max<int64_t>(p->n_items, 1);
  double* partials = ctx_reduce_buffer(ctx, (size_t)n);
  if (p->n_items == 0) cuda_check(cudaMemsetAsync(partials, 0, sizeof(double), ctx->stream), "memset");
  cuda_check(launch_energy_partials(ctx, A->data, B->data, p->d_blocks, p->d_items, p->n_items, partials),
             "energy kernel");
  cuda_check(launch_reduce_final(ctx, partials, n, alpha, 0, out_device), "reduce kernel");
}

void run_norm(tamm_ctx* ctx, const tamm_tensor* t, double* out_device) {
  if (!t) throw Error(TAMM_EINVAL, "norm: null tensor");
  require_data(t, "norm");
  const int64_t parts = std::max<int64_t>(1, std::min<int64_t>((t->n_elems + 8191) / 8192, 4L * ctx->sm_count * 8));
  double* partials = ctx_reduce_buffer(ctx, (size_t)parts);
  if (t->n_elems == 0) cuda_check(cudaMemsetAsync(partials, 0, sizeof(double), ctx->stream), "memset");
  else cuda_check(launch_sumsq_partials(ctx, t->data, t->n_elems, partials, parts), "norm kernel");
  cuda_check(launch_reduce_final(ctx, partials, parts, 1.0, 1, out_device), "reduce kernel");
}

// -------------------------------------------------------- contraction plan

ContractLayout::ContractLayout(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A,
                               const char* la, const tamm_tensor* B, const char* lb) {
  if (!C || !A || !B || !lc || !la || !lb) throw Error(TAMM_EINVAL, "contract: null argument");
  c = C;
  L.add(C, lc, 0, "contract");
  L.add(A, la, 1, "contract");
  L.add(B, lb, 2, "contract");
  for (int i = 0; i < L.n; ++i) {
    const bool c = L.pos[0][i] >= 0, a = L.pos[1][i] >= 0, b = L.pos[2][i] >= 0;
    if (c && a == b)
      throw Error(TAMM_EINVAL, "contract: output label '%c' must appear in exactly one input", L.name[i]);
    if (!c && !(a && b)) throw Error(TAMM_EINVAL, "contract: summed label '%c' must appear in both inputs", L.name[i]);
  }
  // left operand: the one holding C's first label
  swap = L.pos[2][L.find(lc[0])] >= 0;
  left = swap ? B : A;
  right = swap ? A : B;
  const char* ll = swap ? lb : la;
  const char* lr = swap ? la : lb;
  label_left = ll;
  label_right = lr;
  for (const char* p = lc; *p; ++p) (strchr(ll, *p) ? free_left : free_right) += *p;
  for (const char* p = ll; *p; ++p)
    if (!strchr(lc, *p)) summed += *p;
  need_left = free_left + summed;
  need_right = summed + free_right;
  out_gemm = free_left + free_right;
  label_c = lc;
  auto perm_of = [](const std::string& need, const char* have, int* perm) {
    for (size_t m = 0; m < need.size(); ++m) perm[m] = (int)(strchr(have, need[m]) - have);
  };
  int perm[kMaxModes];
  if (need_left != ll) {
    perm_of(need_left, ll, perm);
    left_perm = make_permuted_tensor(*left, perm);
  }
  if (need_right != lr) {
    perm_of(need_right, lr, perm);
    right_perm = make_permuted_tensor(*right, perm);
  }
  if (out_gemm != lc) {
    perm_of(out_gemm, lc, perm);
    out_perm = make_permuted_tensor(*C, perm);
  }
  (void)ctx;
  enumerate();
}

void ContractLayout::enumerate() {
  const tamm_tensor& O = out_perm ? *out_perm : *out_tensor_c();
  const tamm_tensor& Lt = left_perm ? *left_perm : *left;
  const tamm_tensor& Rt = right_perm ? *right_perm : *right;
  const int nfl = (int)free_left.size(), nfr = (int)free_right.size(), nk = (int)summed.size();
  const tamm_space* ksp[kMaxModes];
  int64_t nkt = 1;
  for (int k = 0; k < nk; ++k) {
    ksp[k] = Lt.sp[nfl + k];
    nkt *= ksp[k]->n_tiles;
  }
  flops = 0.0;
  groups.clear();
  tasks.clear();
  for (int64_t ob = 0; ob < O.n_blocks; ++ob) {
    const int64_t* ot = &O.tiles[(size_t)(ob * O.nm)];
    Group g;
    g.out_block = ob;
    g.M = g.N = 1;
    for (int m = 0; m < nfl; ++m) g.M *= O.sp[m]->size[(size_t)ot[m]];
    for (int m = 0; m < nfr; ++m) g.N *= O.sp[nfl + m]->size[(size_t)ot[nfl + m]];
    g.task_begin = (int64_t)tasks.size();
    int64_t lt[kMaxModes], rt[kMaxModes], kt[kMaxModes];
    for (int m = 0; m < nfl; ++m) lt[m] = ot[m];
    for (int m = 0; m < nfr; ++m) rt[nk + m] = ot[nfl + m];
    for (int64_t lin = 0; lin < nkt; ++lin) {
      int64_t r = lin;
      for (int k = nk - 1; k >= 0; --k) {
        kt[k] = r % ksp[k]->n_tiles;
        r /= ksp[k]->n_tiles;
      }
      int64_t K = 1;
      for (int k = 0; k < nk; ++k) {
        lt[nfl + k] = kt[k];
        rt[k] = kt[k];
        K *= ksp[k]->size[(size_t)kt[k]];
      }
      const int64_t lb = Lt.find(lt), rb = Rt.find(rt);
      if (lb < 0 || rb < 0) continue;
      tasks.push_back({lb, rb, K});
      flops += 2.0 * (double)g.M * (double)g.N * (double)K;
    }
    g.task_end = (int64_t)tasks.size();
    groups.push_back(g);
  }
}

double contract_flops(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                      const tamm_tensor* B, const char* lb) {
  ContractLayout lay(ctx, C, lc, A, la, B, lb);
  return lay.flops;
}

// ------------------------------------------------------------ FP64 GEMM path

struct ContractF64Plan : Plan {
  ContractLayout lay;
  std::unique_ptr<AddPlan> perm_left, perm_right, perm_out;
  GemmGroup* d_groups = nullptr;
  GemmTask* d_tasks = nullptr;
  GemmItem* d_items = nullptr;
  int64_t n_items = 0;
  size_t off_l = 0, off_r = 0, off_x = 0, scratch_bytes = 0;

  ContractF64Plan(tamm_ctx* c, const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                  const tamm_tensor* B, const char* lb)
      : Plan(c), lay(c, C, lc, A, la, B, lb) {
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    if (lay.left_perm) {
      const char* ls[1] = {lay.label_left.c_str()};
      perm_left.reset(new AddPlan(c, *lay.left_perm, lay.need_left.c_str(), *lay.left, 1, ls));
      off_l = scratch_bytes;
      scratch_bytes += align((size_t)lay.left_perm->n_elems * 8);
    }
    if (lay.right_perm) {
      const char* ls[1] = {lay.label_right.c_str()};
      perm_right.reset(new AddPlan(c, *lay.right_perm, lay.need_right.c_str(), *lay.right, 1, ls));
      off_r = scratch_bytes;
      scratch_bytes += align((size_t)lay.right_perm->n_elems * 8);
    }
    if (lay.out_perm) {
      const char* ls[1] = {lay.out_gemm.c_str()};
      perm_out.reset(new AddPlan(c, *C, lay.label_c.c_str(), *lay.out_perm, 1, ls));
      off_x = scratch_bytes;
      scratch_bytes += align((size_t)lay.out_perm->n_elems * 8);
    }
    const tamm_tensor& O = lay.out_perm ? *lay.out_perm : *C;
    const tamm_tensor& Lt = lay.left_perm ? *lay.left_perm : *lay.left;
    const tamm_tensor& Rt = lay.right_perm ? *lay.right_perm : *lay.right;
    std::vector<GemmGroup> groups;
    std::vector<GemmTask> tasks;
    std::vector<GemmItem> items;
    for (const auto& g : lay.groups) {
      if (g.M > (1 << 30) || g.N > (1 << 30)) throw Error(TAMM_EUNSUPPORTED, "contract: block too large");
      GemmGroup gg;
      gg.c_off = O.off[(size_t)g.out_block];
      gg.M = (int32_t)g.M;
      gg.N = (int32_t)g.N;
      gg.task_begin = (int32_t)tasks.size();
      for (int64_t t = g.task_begin; t < g.task_end; ++t) {
        const auto& tk = lay.tasks[(size_t)t];
        tasks.push_back({Lt.off[(size_t)tk.left_block], Rt.off[(size_t)tk.right_block], (int32_t)tk.K, 0});
      }
      gg.task_end = (int32_t)tasks.size();
      const int32_t gi = (int32_t)groups.size();
      groups.push_back(gg);
      for (int32_t m0 = 0; m0 < gg.M; m0 += kGemmTileM)
        for (int32_t n0 = 0; n0 < gg.N; n0 += kGemmTileN) items.push_back({gi, m0, n0, 0});
    }
    n_items = (int64_t)items.size();
    d_groups = upload(groups);
    d_tasks = upload(tasks);
    d_items = upload(items);
  }
};

static void check_contract_args(const tamm_tensor* C, const tamm_tensor* A, const tamm_tensor* B, double beta) {
  if (!C || !A || !B) throw Error(TAMM_EINVAL, "contract: null tensor");
  if (beta != 0.0 && beta != 1.0) throw Error(TAMM_EINVAL, "contract: beta must be 0 (=) or 1 (+=)");
  if (C == A || C == B || (C->data && (C->data == A->data || C->data == B->data)))
    throw Error(TAMM_EINVAL, "contract: output aliases an input");
  require_data(C, "contract");
  require_data(A, "contract");
  require_data(B, "contract");
}

void run_contract(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A,
                  const char* la, const tamm_tensor* B, const char* lb, int precision, int slices) {
  if (A && B && (A->lambda || B->lambda)) {
    run_contract_lambda(ctx, alpha, C, lc, beta, A, la, B, lb, precision, slices);
    return;
  }
  check_contract_args(C, A, B, beta);
  if (precision == TAMM_PREC_OZAKI_I8)
    throw Error(TAMM_EUNSUPPORTED, "INT8 slices: sm_103a has no tcgen05 kind::i8 tensor-core product");
  if (precision == TAMM_PREC_OZAKI_BF16) {
    run_contract_ozaki(ctx, alpha, C, lc, beta, A, la, B, lb, slices, false);
    return;
  }
  if (precision == TAMM_PREC_BF16X3) {
    if (slices != 0 && slices != 3) throw Error(TAMM_EINVAL, "bf16x3 uses exactly three slices");
    run_contract_ozaki(ctx, alpha, C, lc, beta, A, la, B, lb, 3, true);
    return;
  }
  if (precision != TAMM_PREC_F64) throw Error(TAMM_EINVAL, "contract: unknown precision %d", precision);
  const std::string key = "f64|" + tid(C) + "|" + lc + "|" + tid(A) + "|" + la + "|" + tid(B) + "|" + lb;
  ContractF64Plan* p = cached<ContractF64Plan>(ctx, key, C, lc, A, la, B, lb);
  char* scratch = p->scratch_bytes ? (char*)ctx_scratch(ctx, p->scratch_bytes) : nullptr;
  const double one = 1.0;
  const double* lp = p->lay.swap ? B->data : A->data;
  const double* rp = p->lay.swap ? A->data : B->data;
  if (p->perm_left) {
    double* dst = (double*)(scratch + p->off_l);
    p->perm_left->run(dst, lp, 0.0, &one);
    lp = dst;
  }
  if (p->perm_right) {
    double* dst = (double*)(scratch + p->off_r);
    p->perm_right->run(dst, rp, 0.0, &one);
    rp = dst;
  }
  double* out = p->perm_out ? (double*)(scratch + p->off_x) : C->data;
  cuda_check(launch_gemm_f64(ctx, lp, rp, out, p->d_groups, p->d_tasks, p->d_items, p->n_items, alpha,
                             p->perm_out ? 0.0 : beta),
             "fp64 gemm kernel");
  if (p->perm_out) p->perm_out->run(C->data, out, beta, &one);
}

}  // namespace tamm
