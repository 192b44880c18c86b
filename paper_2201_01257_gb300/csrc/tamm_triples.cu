// Perturbative triples correction E(T) of CCSD(T) (Sec. IV.B, Eqs. cc14, tensort, tensort2), fused to
// a scalar.
//
// For an occupied triple i<j<k the eighteen terms of W = <Phi_ijk^abc|V_N T2|Phi> are three signed
// permutations of one array (the signs of Eq. tensort absorbed by the antisymmetry of the inputs):
//
//   U[x,y,z] = sum over the cyclic rotations (p,q,r) of (i,j,k) of
//              sum_m T2[x,y,m,r] Vooov[p,q,m,z]  +  sum_e Vvovv[e,p,y,x] T2[e,z,q,r],
//   W[a,b,c] = U[a,b,c] - U[a,c,b] + U[b,c,a].
//
// U of a triple is one block-sparse accumulation per output block (x-tile, y-tile, z-tile), rows
// (x,y) and columns z: six block pairs (three summed over an occupied tile m, three over a virtual
// tile e) in fixed order.  They run on the library's block GEMM kernels: the FP64 kernel, or the
// split-precision tcgen05 kernel whose operand images are sliced once per evaluation.  U exists only
// for one batch of triples (a workspace of bounded size); the fused kernel below then forms W, Y and
// the denominators for every a<b<c of every spin-allowed tile triple and reduces (W + Y) W / D to one
// FP64 partial per warp of each work item; the partials are summed in a fixed order.
#include <algorithm>
#include <array>
#include <cstring>
#include <initializer_list>
#include <string>
#include <memory>
#include <vector>

#include "ozaki.h"
#include "tamm_contract.h"
#include "tamm_plan.h"
#include "tamm_triples.h"

namespace tamm {

// ---------------------------------------------------------------- device

namespace {

// One fused work item: occupied triple n = (i,j,k) and virtual tile triple ta <= tb <= tc.
struct TriplesItem {
  int64_t u_off[3];    // U blocks (ta,tb,tc), (ta,tc,tb), (tb,tc,ta) in the batch workspace
  int64_t voo_off[9];  // Voovv blocks [pair P][virtual pair Q] (-1: not stored); P: ij, ik, jk; Q: ab, ac, bc
  int64_t t1_off[9];   // T1 blocks [virtual v][occupied o] (-1: not stored); v: a, b, c; o: i, j, k
  int32_t pair_pre[3]; // in-block prefix (p_l * |tq| + q_l) of each occupied pair in Voovv
  int32_t occ_loc[3];  // i, j, k inside their tiles (T1 blocks are row-major (virtual, occupied))
  int32_t occ_tsz[3];  // their tile sizes
  int32_t occ[3];      // i, j, k (orbital energies)
  int32_t vlo[3], vn[3];  // offsets and sizes of ta, tb, tc
  int32_t a_begin, a_end;  // the item's range of a inside ta (a tile triple is split so CTAs carry similar work)
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- double-float arithmetic: a value is hi + lo, two FP32 numbers with |lo| <= ulp(hi) / 2, about 48
// significant bits.  GB300 issues FP32 operations at 64 times its FP64 rate, so the fused energy
// evaluates W, Y, the denominator and (W + Y) W / D in this form.  Error-free transformations
// (Knuth's TwoSum, Dekker's FastTwoSum, the FMA product error) with explicitly rounded operations, so
// that no multiply-add contraction changes them.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// x / d: quotient of the leading parts, then one correction from the double-float residual x - q d.
__device__ __forceinline__ df df_div(df x, df d) {
  const float r = __frcp_rn(d.hi);
  const float q1 = __fmul_rn(x.hi, r);
  const df res = df_add(x, df_neg(df_mul({q1, 0.0f}, d)));
  const float q2 = __fmul_rn(res.hi, r);
  return fast_two_sum(q1, q2);
}
// A double split into hi (its leading 24 bits, truncated) and lo (the rest, rounded to 24 bits), built from
// the bit pattern with integer operations (no FP64 instruction).  Magnitudes below 2^-74 read as zero;
// the inputs here are amplitudes, integrals and orbital energies, far inside the range.
__device__ __forceinline__ df df_from(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  if (E < -74) return {0.0f, 0.0f};
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const unsigned long long m = b & ((1ull << 52) - 1);
  const float hi = __uint_as_float(sign | (uint32_t)(E + 127) << 23 | (uint32_t)(m >> 29));
  const float rem = __uint2float_rn((uint32_t)(m & ((1u << 29) - 1)));  // the low 29 mantissa bits
  const float lo = __fmul_rn(rem, __uint_as_float((uint32_t)(E - 52 + 127) << 23));
  return {hi, sign ? -lo : lo};
}

// Double-float copies of the fused kernel's small inputs (V_oovv, T1, orbital energies).
__global__ void to_df_kernel(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const df v = df_from(x[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}

__device__ __forceinline__ df ld(const float2* p, int64_t i) {
  const float2 v = p[i];
  return {v.x, v.y};
}

constexpr int kEnergyB = 16;     // consecutive b per unit of the fused energy kernel
constexpr int kEnergyWarps = 8;  // warps per CTA of the fused energy kernel: one partial each

// One item per CTA.  The item's (a, b, c) are cut into units of four consecutive a (one 32-byte sector of
// U[b,c,a]), one c and a run of kEnergyB consecutive b, the units spread over the threads with c fastest,
// so U[a,b,c] is read coalesced across the warp (consecutive c), U[a,c,b] along one row per thread and
// U[b,c,a] in whole sectors, and every thread carries about the same number of (a, b, c) (a thread that
// owned all b of its (a, c) left most of the CTA waiting on the longest walk).  Y of Eq. tensort2 is
// nine products: each T1 factor carries its pair's sign (pairs (ij)k, (ik)j, (jk)i: +, -, +) and the
// virtual split's (ab|c +, ac|b -, bc|a +).  Double-float arithmetic; each warp's sum goes to
// partials[blockIdx.x * kEnergyWarps + warp] in FP64.
__global__ void __launch_bounds__(256) triples_energy_kernel(const double* __restrict__ U,
                                                             const TriplesItem* __restrict__ items,
                                                             const float2* __restrict__ voo,
                                                             const float2* __restrict__ t1,
                                                             const float2* __restrict__ eps_o,
                                                             const float2* __restrict__ eps_v,
                                                             double* __restrict__ partials) {
  const TriplesItem& it = items[blockIdx.x];
  const int na = it.vn[0], nb = it.vn[1], nc = it.vn[2];
  const int a0 = it.vlo[0], b0 = it.vlo[1], c0 = it.vlo[2];
  const df e_occ = df_add(df_add(ld(eps_o, it.occ[0]), ld(eps_o, it.occ[1])), ld(eps_o, it.occ[2]));
  const double* U1 = U + it.u_off[0];
  const double* U2 = U + it.u_off[1];
  const double* U3 = U + it.u_off[2];
  const int q0 = it.a_begin / 4, nquad = (it.a_end + 3) / 4 - q0;
  // the single occupied orbital of pair P ((ij) -> k, (ik) -> j, (jk) -> i) and the pair's sign
  constexpr int kSingle[3] = {2, 1, 0};
  constexpr float kSign[3] = {1.0f, -1.0f, 1.0f};
  auto t1s = [&](int v, int P, int l) -> df {  // sign_P * T1[virtual v (local index l), single(P)]
    const int o = kSingle[P];
    const int64_t off = it.t1_off[v * 3 + o];
    if (off < 0) return {0.0f, 0.0f};
    const df x = ld(t1, off + (int64_t)l * it.occ_tsz[o] + it.occ_loc[o]);
    return {kSign[P] * x.hi, kSign[P] * x.lo};
  };
  df acc = {0.0f, 0.0f};
  const int nbr = (nb + kEnergyB - 1) / kEnergyB;  // runs of b
  for (int u = threadIdx.x; u < nquad * nbr * nc; u += blockDim.x) {
    const int cl = u % nc, r = u / nc, br = r % nbr, q = q0 + r / nbr;
    const int c = c0 + cl;
    const int bl0 = br * kEnergyB, bl1 = min(nb, bl0 + kEnergyB);
    if (b0 + bl0 >= c || b0 + bl1 - 1 <= a0 + 4 * q) continue;  // no b of this run lies in (a, c)
    const df e_c = df_add(e_occ, df_neg(ld(eps_v, c)));
    df tc[3];  // term v_P[a,b] t1[c]
#pragma unroll
    for (int P = 0; P < 3; ++P) tc[P] = t1s(2, P, cl);
    for (int al = 4 * q; al < min(it.a_end, 4 * q + 4); ++al) {
      const int a = a0 + al;
      if (a >= c) break;
      const df e_ac = df_add(e_c, df_neg(ld(eps_v, a)));
      df ta[3], vac[3];  // term v_P[b,c] t1[a];  v_P[a,c]
#pragma unroll
      for (int P = 0; P < 3; ++P) {
        ta[P] = t1s(0, P, al);
        const int64_t ov = it.voo_off[P * 3 + 1];
        vac[P] = ov >= 0 ? ld(voo, ov + ((int64_t)it.pair_pre[P] * na + al) * nc + cl) : df{0.0f, 0.0f};
      }
      for (int bl = bl0; bl < bl1; ++bl) {
        const int b = b0 + bl;
        if (b <= a) continue;
        if (b >= c) break;
        const df w = df_add(df_add(df_from(U1[((int64_t)al * nb + bl) * nc + cl]),
                                   df_neg(df_from(U2[((int64_t)al * nc + cl) * nb + bl]))),
                            df_from(U3[((int64_t)bl * nc + cl) * na + al]));
        df y = {0.0f, 0.0f};
#pragma unroll
        for (int P = 0; P < 3; ++P) {
          const int64_t oab = it.voo_off[P * 3 + 0], obc = it.voo_off[P * 3 + 2];
          const df vab = oab >= 0 ? ld(voo, oab + ((int64_t)it.pair_pre[P] * na + al) * nb + bl) : df{0.0f, 0.0f};
          const df vbc = obc >= 0 ? ld(voo, obc + ((int64_t)it.pair_pre[P] * nb + bl) * nc + cl) : df{0.0f, 0.0f};
          const df tb = t1s(1, P, bl);
          y = df_add(y, df_mul(vab, tc[P]));           // + v_P[a,b] t1[c]
          y = df_add(y, df_neg(df_mul(vac[P], tb)));   // - v_P[a,c] t1[b]
          y = df_add(y, df_mul(vbc, ta[P]));           // + v_P[b,c] t1[a]
        }
        const df d = df_add(e_ac, df_neg(ld(eps_v, b)));  // e_i + e_j + e_k - e_a - e_b - e_c
        acc = df_add(acc, df_div(df_mul(df_add(w, y), w), d));
      }
    }
  }
  // one partial per warp (no CTA-wide barrier: a warp that is done leaves instead of waiting for the
  // CTA's longest walk); the partials are summed in a fixed order afterwards
  double v = (double)acc.hi + (double)acc.lo;
  v = warp_sum(v);
  if (threadIdx.x % 32 == 0) partials[(int64_t)blockIdx.x * kEnergyWarps + threadIdx.x / 32] = v;
}

// out[t] = sum of the partials of items seg[t] .. seg[t+1] (kEnergyWarps each) in order (one thread per triple).
__global__ void triples_segment_kernel(const double* __restrict__ partials, const int64_t* __restrict__ seg,
                                       int64_t n, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int64_t i = seg[t] * kEnergyWarps; i < seg[t + 1] * kEnergyWarps; ++i) s += partials[i];
  out[t] = s;
}

}  // namespace

// ------------------------------------------------------------------ host

namespace {

struct Occ {
  int32_t tile, loc;
};

constexpr int32_t kEnergyRows = 8;  // values of a per fused energy work item

// Spin-allowed output blocks (tx,ty,tz) of U for one total spin of the occupied triple, packed.
struct BlockTable {
  std::vector<int32_t> tx, ty, tz;
  std::vector<int64_t> off;  // element offsets, n + 1 entries
  std::vector<int32_t> index;  // (tx * nt + ty) * nt + tz -> block or -1
};

int64_t block_find(const tamm_tensor& T, std::initializer_list<int64_t> tiles) {
  int64_t tt[kMaxModes];
  int m = 0;
  for (int64_t x : tiles) tt[m++] = x;
  return T.find(tt);
}

}  // namespace

struct TriplesPlan : Plan {
  // spaces and inputs
  const tamm_space* O = nullptr;
  const tamm_space* V = nullptr;
  int64_t no = 0, nv = 0;
  int nto = 0, ntv = 0;
  std::vector<Occ> occ;
  std::vector<std::array<int32_t, 3>> triples;
  BlockTable tables[7];  // by total spin + 3 (odd values only)
  int64_t n_batches = 0;
  std::vector<int64_t> batch_triple0;  // first triple of each batch (n_batches + 1)
  std::vector<int64_t> triple_ws;      // workspace offset of each triple inside its batch
  int64_t ws_elems = 0;                // largest batch workspace (doubles)
  double gemm_flops = 0.0;

  // GEMM-order copies (both precisions): Tq[r,x,y,m] = T2[x,y,m,r], Vp[p,x,y,e] = Vvovv[e,p,y,x],
  // Tz[q,r,e,z] = T2[e,z,q,r]; Vooov is read in place.
  std::unique_ptr<tamm_tensor> Tq, Vp, Tz;
  std::unique_ptr<AddPlan> copy_q, copy_p, copy_z;

  // FP64 path
  std::vector<GemmGroup> fgroups_q, fgroups_z;
  std::vector<GemmTask> ftasks_q, ftasks_z;
  std::vector<GemmItem> fitems;
  std::vector<int64_t> fitem_begin;  // per batch
  GemmGroup *d_fgroups_q = nullptr, *d_fgroups_z = nullptr;
  GemmTask *d_ftasks_q = nullptr, *d_ftasks_z = nullptr;
  GemmItem* d_fitems = nullptr;

  // split path (built on first use for a slice count and tile policy)
  int oz_S = 0, oz_policy = -1;
  bool oz_shared = false;
  int64_t slots_a = 0, slots_b = 0;  // shared scaling: rows (x,y) of each (x-tile, y-tile), columns z of each z-tile
  std::vector<SliceBlock> rec[4];  // A from Tq, A from Vp, B from Vooov, B from Tz
  std::vector<SliceItem> sitems[4];
  int warps[4] = {8, 8, 8, 8}, kbuf[4] = {2, 2, 2, 2};
  SliceBlock* d_rec[4] = {};
  SliceItem* d_sitems[4] = {};
  int64_t a_bytes = 0, b_bytes = 0, a_rows = 0, b_rows = 0;
  std::vector<int64_t> oitem_begin;  // per batch
  OzGroup* d_ogroups = nullptr;
  OzTask* d_otasks = nullptr;
  OzItem* d_oitems = nullptr;

  // fused energy
  std::vector<int64_t> eitem_begin;  // per batch
  TriplesItem* d_eitems = nullptr;
  int64_t n_eitems = 0;
  int64_t* d_seg = nullptr;  // per triple: its first item (n_triples + 1)

  TriplesPlan(tamm_ctx* c, const tamm_tensor& T2, const tamm_tensor& T1, const tamm_tensor& Vo, const tamm_tensor& Vv,
              const tamm_tensor& Voo, int64_t workspace_bytes, bool device)
      : Plan(c) {
    V = T2.sp[0];
    O = T2.sp[2];
    no = O->n;
    nv = V->n;
    nto = O->n_tiles;
    ntv = V->n_tiles;
    for (int t = 0; t < nto; ++t)
      for (int64_t l = 0; l < O->size[(size_t)t]; ++l) occ.push_back({(int32_t)t, (int32_t)l});
    for (int32_t i = 0; i < no; ++i)
      for (int32_t j = i + 1; j < no; ++j)
        for (int32_t k = j + 1; k < no; ++k) triples.push_back({i, j, k});
    // U blocks: spin(x) + spin(y) + spin(z) = spin(i) + spin(j) + spin(k)
    for (int s = -3; s <= 3; ++s) {
      BlockTable& bt = tables[s + 3];
      bt.index.assign((size_t)ntv * ntv * ntv, -1);
      bt.off.assign(1, 0);
      for (int x = 0; x < ntv; ++x)
        for (int y = 0; y < ntv; ++y)
          for (int z = 0; z < ntv; ++z) {
            if (V->spin[(size_t)x] + V->spin[(size_t)y] + V->spin[(size_t)z] != s) continue;
            bt.index[(size_t)((x * ntv + y) * ntv + z)] = (int32_t)bt.tx.size();
            bt.tx.push_back(x);
            bt.ty.push_back(y);
            bt.tz.push_back(z);
            bt.off.push_back(bt.off.back() + V->size[(size_t)x] * V->size[(size_t)y] * V->size[(size_t)z]);
          }
    }
    // batches of consecutive triples whose U fit the workspace
    const int64_t budget = std::max<int64_t>(1, (workspace_bytes > 0 ? workspace_bytes : (int64_t(1) << 30)) / 8);
    batch_triple0.push_back(0);
    int64_t used = 0;
    triple_ws.resize(triples.size());
    for (size_t n = 0; n < triples.size(); ++n) {
      const int64_t need = table_of(n).off.back();
      if (used > 0 && used + need > budget) {
        batch_triple0.push_back((int64_t)n);
        used = 0;
      }
      triple_ws[n] = used;
      used += need;
      ws_elems = std::max(ws_elems, used);
    }
    batch_triple0.push_back((int64_t)triples.size());
    n_batches = (int64_t)batch_triple0.size() - 1;
    if (triples.empty()) n_batches = 0;

    // GEMM-order copies (block tables only on a host-only context)
    const int pq[4] = {3, 0, 1, 2}, pp[4] = {1, 3, 2, 0}, pz[4] = {2, 3, 0, 1};
    Tq = make_permuted_tensor(T2, pq);
    Vp = make_permuted_tensor(Vv, pp);
    Tz = make_permuted_tensor(T2, pz);
    build_fp64_tasks(T2, Vo, Vv);
    if (device) {
      alloc_copy(Tq);
      alloc_copy(Vp);
      alloc_copy(Tz);
      const char* lq[1] = {"abcd"};
      copy_q.reset(new AddPlan(c, *Tq, "dabc", T2, 1, lq));
      copy_p.reset(new AddPlan(c, *Vp, "bdca", Vv, 1, lq));
      copy_z.reset(new AddPlan(c, *Tz, "cdab", T2, 1, lq));
      d_fgroups_q = upload(fgroups_q);
      d_fgroups_z = upload(fgroups_z);
      d_ftasks_q = upload(ftasks_q.empty() ? std::vector<GemmTask>(1) : ftasks_q);
      d_ftasks_z = upload(ftasks_z.empty() ? std::vector<GemmTask>(1) : ftasks_z);
      d_fitems = upload(fitems);
      build_energy_items(T1, Voo);
    }
  }

  ~TriplesPlan() override {
    for (auto* T : {Tq.get(), Vp.get(), Tz.get()})
      if (T && T->owned) ctx_free(ctx, T->data, T->owned_bytes);
  }

  const BlockTable& table_of(size_t n) const {
    const auto& t = triples[n];
    const int s = O->spin[(size_t)occ[(size_t)t[0]].tile] + O->spin[(size_t)occ[(size_t)t[1]].tile] +
                  O->spin[(size_t)occ[(size_t)t[2]].tile];
    return tables[s + 3];
  }

  void alloc_copy(std::unique_ptr<tamm_tensor>& T) {
    const size_t bytes = (size_t)std::max<int64_t>(T->n_elems, 1) * 8;
    T->data = (double*)ctx_alloc(ctx, bytes);
    T->owned = true;
    T->owned_bytes = bytes;
  }

  // The six block pairs of every (triple, U block), in the order Q (occupied m) then Z (virtual e),
  // rotations (i,j,k), (j,k,i), (k,i,j); `visit(is_z, tile m|e, p, q, r)` for each stored pair.
  template <class F>
  void for_pairs(const std::array<int32_t, 3>& t, int tx, int ty, int tz, const tamm_tensor& T2,
                 const tamm_tensor& Vo, const tamm_tensor& Vv, F&& visit) const {
    const int32_t rot[3][3] = {{t[0], t[1], t[2]}, {t[1], t[2], t[0]}, {t[2], t[0], t[1]}};
    for (int r3 = 0; r3 < 3; ++r3) {
      const int32_t p = rot[r3][0], q = rot[r3][1], r = rot[r3][2];
      const int tp = occ[(size_t)p].tile, tq = occ[(size_t)q].tile, tr = occ[(size_t)r].tile;
      for (int tm = 0; tm < nto; ++tm)
        if (block_find(T2, {tx, ty, tm, tr}) >= 0 && block_find(Vo, {tp, tq, tm, tz}) >= 0) visit(false, tm, p, q, r);
    }
    for (int r3 = 0; r3 < 3; ++r3) {
      const int32_t p = rot[r3][0], q = rot[r3][1], r = rot[r3][2];
      const int tp = occ[(size_t)p].tile, tq = occ[(size_t)q].tile, tr = occ[(size_t)r].tile;
      for (int te = 0; te < ntv; ++te)
        if (block_find(Vv, {te, tp, ty, tx}) >= 0 && block_find(T2, {te, tz, tq, tr}) >= 0) visit(true, te, p, q, r);
    }
  }

  void build_fp64_tasks(const tamm_tensor& T2, const tamm_tensor& Vo, const tamm_tensor& Vv) {
    fitem_begin.push_back(0);
    for (int64_t bch = 0; bch < n_batches; ++bch) {
      for (int64_t n = batch_triple0[(size_t)bch]; n < batch_triple0[(size_t)bch + 1]; ++n) {
        const auto& t = triples[(size_t)n];
        const BlockTable& bt = table_of((size_t)n);
        for (size_t g = 0; g < bt.tx.size(); ++g) {
          const int tx = bt.tx[g], ty = bt.ty[g], tz = bt.tz[g];
          const int64_t nx = V->size[(size_t)tx], ny = V->size[(size_t)ty], nz = V->size[(size_t)tz];
          GemmGroup gq{triple_ws[(size_t)n] + bt.off[g], (int32_t)(nx * ny), (int32_t)nz, (int32_t)ftasks_q.size(), 0};
          GemmGroup gz = gq;
          gz.task_begin = (int32_t)ftasks_z.size();
          for_pairs(t, tx, ty, tz, T2, Vo, Vv, [&](bool is_z, int tk, int32_t p, int32_t q, int32_t r) {
            const Occ op = occ[(size_t)p], oq = occ[(size_t)q], orr = occ[(size_t)r];
            const int64_t nk = is_z ? V->size[(size_t)tk] : O->size[(size_t)tk];
            gemm_flops += 2.0 * (double)(nx * ny) * (double)nz * (double)nk;
            if (!is_z) {
              const int64_t ba = block_find(*Tq, {orr.tile, tx, ty, tk});
              const int64_t bb = block_find(Vo, {op.tile, oq.tile, tk, tz});
              ftasks_q.push_back({Tq->off[(size_t)ba] + orr.loc * nx * ny * nk,
                                  Vo.off[(size_t)bb] + ((int64_t)op.loc * O->size[(size_t)oq.tile] + oq.loc) * nk * nz,
                                  (int32_t)nk, 0});
            } else {
              const int64_t ba = block_find(*Vp, {op.tile, tx, ty, tk});
              const int64_t bb = block_find(*Tz, {oq.tile, orr.tile, tk, tz});
              ftasks_z.push_back({Vp->off[(size_t)ba] + op.loc * nx * ny * nk,
                                  Tz->off[(size_t)bb] + ((int64_t)oq.loc * O->size[(size_t)orr.tile] + orr.loc) * nk * nz,
                                  (int32_t)nk, 0});
            }
          });
          gq.task_end = (int32_t)ftasks_q.size();
          gz.task_end = (int32_t)ftasks_z.size();
          const int32_t gi = (int32_t)fgroups_q.size();
          fgroups_q.push_back(gq);
          fgroups_z.push_back(gz);
          for (int32_t m0 = 0; m0 < gq.M; m0 += kGemmTileM)
            for (int32_t n0 = 0; n0 < gq.N; n0 += kGemmTileN) fitems.push_back({gi, m0, n0, 0});
        }
      }
      fitem_begin.push_back((int64_t)fitems.size());
    }
  }

  void build_energy_items(const tamm_tensor& T1, const tamm_tensor& Voo) {
    std::vector<TriplesItem> items;
    std::vector<int64_t> seg;
    eitem_begin.push_back(0);
    for (int64_t bch = 0; bch < n_batches; ++bch) {
      for (int64_t n = batch_triple0[(size_t)bch]; n < batch_triple0[(size_t)bch + 1]; ++n) {
        seg.push_back((int64_t)items.size());
        const auto& t = triples[(size_t)n];
        const BlockTable& bt = table_of((size_t)n);
        const Occ o3[3] = {occ[(size_t)t[0]], occ[(size_t)t[1]], occ[(size_t)t[2]]};
        const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int ta = 0; ta < ntv; ++ta)
          for (int tb = ta; tb < ntv; ++tb)
            for (int tc = tb; tc < ntv; ++tc) {
              const int32_t g0 = bt.index[(size_t)((ta * ntv + tb) * ntv + tc)];
              if (g0 < 0) continue;
              const int32_t g1 = bt.index[(size_t)((ta * ntv + tc) * ntv + tb)];
              const int32_t g2 = bt.index[(size_t)((tb * ntv + tc) * ntv + ta)];
              if (g1 < 0 || g2 < 0) throw Error(TAMM_EINVAL, "triples: permuted U block missing");
              TriplesItem it;
              memset(&it, 0, sizeof(it));
              const int64_t base = triple_ws[(size_t)n];
              it.u_off[0] = base + bt.off[(size_t)g0];
              it.u_off[1] = base + bt.off[(size_t)g1];
              it.u_off[2] = base + bt.off[(size_t)g2];
              const int vt[3] = {ta, tb, tc};
              const int vq[3][2] = {{ta, tb}, {ta, tc}, {tb, tc}};
              for (int P = 0; P < 3; ++P) {
                const Occ op = o3[pairs[P][0]], oq = o3[pairs[P][1]];
                it.pair_pre[P] = op.loc * (int32_t)O->size[(size_t)oq.tile] + oq.loc;
                for (int Q = 0; Q < 3; ++Q) {
                  const int64_t b = block_find(Voo, {op.tile, oq.tile, vq[Q][0], vq[Q][1]});
                  it.voo_off[P * 3 + Q] = b >= 0 ? Voo.off[(size_t)b] : -1;
                }
              }
              for (int v = 0; v < 3; ++v)
                for (int o = 0; o < 3; ++o) {
                  const int64_t b = block_find(T1, {vt[v], o3[o].tile});
                  it.t1_off[v * 3 + o] = b >= 0 ? T1.off[(size_t)b] : -1;
                }
              for (int o = 0; o < 3; ++o) {
                it.occ_loc[o] = o3[o].loc;
                it.occ_tsz[o] = (int32_t)O->size[(size_t)o3[o].tile];
                it.occ[o] = t[o];
              }
              for (int v = 0; v < 3; ++v) {
                it.vlo[v] = (int32_t)V->off[(size_t)vt[v]];
                it.vn[v] = (int32_t)V->size[(size_t)vt[v]];
              }
              // a ranges of kEnergyRows (a multiple of 4: whole sectors of U[b,c,a])
              for (int32_t a0 = 0; a0 < it.vn[0]; a0 += kEnergyRows) {
                it.a_begin = a0;
                it.a_end = std::min<int32_t>(it.vn[0], a0 + kEnergyRows);
                items.push_back(it);
              }
            }
      }
      eitem_begin.push_back((int64_t)items.size());
    }
    seg.push_back((int64_t)items.size());
    n_eitems = (int64_t)items.size();
    if (n_eitems > 0x7FFFFFFF) throw Error(TAMM_EUNSUPPORTED, "triples: too many work items");
    d_eitems = upload(items.empty() ? std::vector<TriplesItem>(1) : items);
    d_seg = upload(seg);
  }

  // Split-precision images and tasks for slice count S (kept until another S or policy is asked for).
  void build_split(int S, int policy, bool shared) {
    if (S == oz_S && policy == oz_policy && shared == oz_shared) return;
    oz_S = S;
    oz_policy = policy;
    oz_shared = shared;
    // shared-scaling slots: one per U row (x,y) of each tile pair and one per U column z of each tile
    std::vector<int64_t> base_a((size_t)ntv * ntv), base_b((size_t)ntv);
    slots_a = slots_b = 0;
    for (int x = 0; x < ntv; ++x)
      for (int y = 0; y < ntv; ++y) {
        base_a[(size_t)(x * ntv + y)] = slots_a;
        slots_a += V->size[(size_t)x] * V->size[(size_t)y];
      }
    for (int z = 0; z < ntv; ++z) {
      base_b[(size_t)z] = slots_b;
      slots_b += V->size[(size_t)z];
    }
    for (int s = 0; s < 4; ++s) {
      rec[s].clear();
      sitems[s].clear();
    }
    a_bytes = b_bytes = a_rows = b_rows = 0;
    std::vector<int32_t> ext[4];
    const tamm_tensor& T2q = *Tq;
    // image indices: A_Q (r, tx, ty, tm), A_Z (p, tx, ty, te), B_Q (p, q, tm, tz), B_Z (q, r, te, tz)
    std::vector<int32_t> iaq((size_t)no * ntv * ntv * nto, -1), iaz((size_t)no * ntv * ntv * ntv, -1);
    std::vector<int32_t> ibq((size_t)no * no * nto * ntv, -1), ibz((size_t)no * no * ntv * ntv, -1);
    auto add_rec = [&](int set, int64_t src_off, int64_t rows, int32_t rstride, int64_t K, int32_t kstride,
                       bool is_a, int H, int64_t slot) {
      SliceBlock B;
      memset(&B, 0, sizeof(B));
      B.src_off = src_off;
      B.nr = 1;
      B.nk = 1;
      B.rdim[0] = (int32_t)rows;
      B.rstride[0] = rstride;
      B.kdim[0] = (int32_t)K;
      B.kstride[0] = kstride;
      B.rows = (int32_t)rows;
      B.K = (int32_t)K;
      B.k_tiles = (int32_t)((K + kOzTileK - 1) / kOzTileK);
      B.k_contig = kstride == 1 ? 1 : 0;
      B.k_dense = kstride == 1 ? 1 : 0;
      B.tile_rows = is_a ? kOzTileM : H;
      B.row_tiles = (int32_t)((rows + B.tile_rows - 1) / B.tile_rows);
      B.dst_row0 = 0;
      B.shared_off = slot;
      int64_t& bytes = is_a ? a_bytes : b_bytes;
      int64_t& erow = is_a ? a_rows : b_rows;
      B.tile_off = bytes;
      B.exp_off = erow;
      bytes += (int64_t)B.row_tiles * B.k_tiles * S * B.tile_rows * 32;
      erow += (int64_t)B.row_tiles * B.tile_rows;
      rec[set].push_back(B);
      ext[set].push_back(B.row_tiles * B.tile_rows);
      return (int32_t)(rec[set].size() - 1);
    };
    auto H_of = [&](int tz) { return oz_tile_rows(V->size[(size_t)tz], policy); };
    // A images of every orbital and stored block
    for (int32_t r = 0; r < no; ++r)
      for (int64_t b = 0; b < T2q.n_blocks; ++b) {
        const int64_t* tt = &T2q.tiles[(size_t)(b * 4)];  // (tr, tx, ty, tm)
        if (tt[0] != occ[(size_t)r].tile) continue;
        const int64_t nx = V->size[(size_t)tt[1]], ny = V->size[(size_t)tt[2]], nk = O->size[(size_t)tt[3]];
        iaq[(size_t)(((r * ntv + tt[1]) * ntv + tt[2]) * nto + tt[3])] =
            add_rec(0, T2q.off[(size_t)b] + occ[(size_t)r].loc * nx * ny * nk, nx * ny, (int32_t)nk, nk, 1, true, 0,
                    base_a[(size_t)(tt[1] * ntv + tt[2])]);
      }
    for (int32_t p = 0; p < no; ++p)
      for (int64_t b = 0; b < Vp->n_blocks; ++b) {
        const int64_t* tt = &Vp->tiles[(size_t)(b * 4)];  // (tp, tx, ty, te)
        if (tt[0] != occ[(size_t)p].tile) continue;
        const int64_t nx = V->size[(size_t)tt[1]], ny = V->size[(size_t)tt[2]], nk = V->size[(size_t)tt[3]];
        iaz[(size_t)(((p * ntv + tt[1]) * ntv + tt[2]) * ntv + tt[3])] =
            add_rec(1, Vp->off[(size_t)b] + occ[(size_t)p].loc * nx * ny * nk, nx * ny, (int32_t)nk, nk, 1, true, 0,
                    base_a[(size_t)(tt[1] * ntv + tt[2])]);
      }
    // B images of every ordered occupied pair and stored block
    for (int32_t p = 0; p < no; ++p)
      for (int32_t q = 0; q < no; ++q) {
        if (p == q) continue;
        const Occ op = occ[(size_t)p], oq = occ[(size_t)q];
        for (int tm = 0; tm < nto; ++tm)
          for (int tz = 0; tz < ntv; ++tz) {
            const int64_t b = block_find(*vo_, {op.tile, oq.tile, tm, tz});
            if (b < 0) continue;
            const int64_t nk = O->size[(size_t)tm], nz = V->size[(size_t)tz];
            ibq[(size_t)(((p * no + q) * nto + tm) * ntv + tz)] =
                add_rec(2, vo_->off[(size_t)b] + ((int64_t)op.loc * O->size[(size_t)oq.tile] + oq.loc) * nk * nz, nz, 1,
                        nk, (int32_t)nz, false, H_of(tz), base_b[(size_t)tz]);
          }
        for (int te = 0; te < ntv; ++te)
          for (int tz = 0; tz < ntv; ++tz) {
            const int64_t b = block_find(*Tz, {op.tile, oq.tile, te, tz});
            if (b < 0) continue;
            const int64_t nk = V->size[(size_t)te], nz = V->size[(size_t)tz];
            ibz[(size_t)(((p * no + q) * ntv + te) * ntv + tz)] =
                add_rec(3, Tz->off[(size_t)b] + ((int64_t)op.loc * O->size[(size_t)oq.tile] + oq.loc) * nk * nz, nz, 1,
                        nk, (int32_t)nz, false, H_of(tz), base_b[(size_t)tz]);
          }
      }
    for (int s = 0; s < 4; ++s) oz_slicing_items(rec[s], ext[s], sitems[s], warps[s], kbuf[s]);
    // groups, tasks and items per batch
    std::vector<OzGroup> groups;
    std::vector<OzTask> tasks;
    std::vector<OzItem> items;
    oitem_begin.assign(1, 0);
    for (int64_t bch = 0; bch < n_batches; ++bch) {
      for (int64_t n = batch_triple0[(size_t)bch]; n < batch_triple0[(size_t)bch + 1]; ++n) {
        const auto& t = triples[(size_t)n];
        const BlockTable& bt = table_of((size_t)n);
        for (size_t g = 0; g < bt.tx.size(); ++g) {
          const int tx = bt.tx[g], ty = bt.ty[g], tz = bt.tz[g];
          const int64_t nx = V->size[(size_t)tx], ny = V->size[(size_t)ty], nz = V->size[(size_t)tz];
          const int H = H_of(tz);
          OzGroup gg;
          memset(&gg, 0, sizeof(gg));
          gg.c_off = triple_ws[(size_t)n] + bt.off[g];
          gg.colmap = -1;
          gg.M = (int32_t)(nx * ny);
          gg.N = (int32_t)nz;
          gg.n_tile = H;
          gg.nsplit = 1;
          gg.shared = shared ? 1 : 0;
          gg.task_begin = (int32_t)tasks.size();
          for_pairs(t, tx, ty, tz, *t2_, *vo_, *vv_, [&](bool is_z, int tk, int32_t p, int32_t q, int32_t r) {
            int32_t ia, ib, sa, sb;
            if (!is_z) {
              ia = iaq[(size_t)(((r * ntv + tx) * ntv + ty) * nto + tk)];
              ib = ibq[(size_t)(((p * no + q) * nto + tk) * ntv + tz)];
              sa = 0;
              sb = 2;
            } else {
              ia = iaz[(size_t)(((p * ntv + tx) * ntv + ty) * ntv + tk)];
              ib = ibz[(size_t)(((q * no + r) * ntv + tk) * ntv + tz)];
              sa = 1;
              sb = 3;
            }
            if (ia < 0 || ib < 0) throw Error(TAMM_EINVAL, "triples: operand image missing");
            const SliceBlock& A = rec[sa][(size_t)ia];
            const SliceBlock& B = rec[sb][(size_t)ib];
            if (A.k_tiles != B.k_tiles) throw Error(TAMM_EINVAL, "triples: K mismatch");
            tasks.push_back({A.tile_off, B.tile_off, A.exp_off, B.exp_off, A.k_tiles, 0});
          });
          gg.task_end = (int32_t)tasks.size();
          const int32_t gi = (int32_t)groups.size();
          groups.push_back(gg);
          const int32_t mts = (gg.M + kOzTileM - 1) / kOzTileM, nts = (gg.N + H - 1) / H;
          for (int32_t mt = 0; mt < mts; ++mt)
            for (int32_t nt = 0; nt < nts; ++nt) items.push_back({gi, mt, nt, -1, gg.task_begin, gg.task_end});
        }
      }
      oitem_begin.push_back((int64_t)items.size());
    }
    for (int s = 0; s < 4; ++s) {
      d_rec[s] = upload(rec[s].empty() ? std::vector<SliceBlock>(1) : rec[s]);
      d_sitems[s] = upload(sitems[s].empty() ? std::vector<SliceItem>(1) : sitems[s]);
    }
    d_ogroups = upload(groups.empty() ? std::vector<OzGroup>(1) : groups);
    d_otasks = upload(tasks.empty() ? std::vector<OzTask>(1) : tasks);
    d_oitems = upload(items.empty() ? std::vector<OzItem>(1) : items);
  }

  // the input tensors the plan was built for (their block tables; data pointers are read per call)
  const tamm_tensor* t2_ = nullptr;
  const tamm_tensor* vo_ = nullptr;
  const tamm_tensor* vv_ = nullptr;
};

namespace {

void check_triples_inputs(const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vo, const tamm_tensor* Vv,
                          const tamm_tensor* Voo) {
  if (!T2 || !T1 || !Vo || !Vv || !Voo) throw Error(TAMM_EINVAL, "triples: null tensor");
  for (const tamm_tensor* X : {T2, T1, Vo, Vv, Voo})
    if (X->lambda) throw Error(TAMM_EUNSUPPORTED, "triples: a lambda tensor has no storage");
  if (T2->nm != 4 || T1->nm != 2 || Vo->nm != 4 || Vv->nm != 4 || Voo->nm != 4)
    throw Error(TAMM_EINVAL, "triples: T2, Vooov, Vvovv, Voovv need 4 modes and T1 2");
  const tamm_space* V = T2->sp[0];
  const tamm_space* O = T2->sp[2];
  if (V == O) throw Error(TAMM_EINVAL, "triples: occupied and virtual spaces must differ");
  const bool ok = T2->sp[1] == V && T2->sp[3] == O && T1->sp[0] == V && T1->sp[1] == O && Vo->sp[0] == O &&
                  Vo->sp[1] == O && Vo->sp[2] == O && Vo->sp[3] == V && Vv->sp[0] == V && Vv->sp[1] == O &&
                  Vv->sp[2] == V && Vv->sp[3] == V && Voo->sp[0] == O && Voo->sp[1] == O && Voo->sp[2] == V &&
                  Voo->sp[3] == V;
  if (!ok) throw Error(TAMM_EINVAL, "triples: tensors must be T2(v,v,o,o), T1(v,o), Vooov(o,o,o,v), Vvovv(v,o,v,v), "
                       "Voovv(o,o,v,v) on one occupied and one virtual space");
  for (const tamm_space* s : {V, O}) {
    int64_t cap = 0;
    for (int t = 0; t < s->n_tiles; ++t) cap = std::max(cap, s->size[(size_t)t]);
    if (cap * cap > (int64_t(1) << 30)) throw Error(TAMM_EUNSUPPORTED, "triples: tiles too large");
  }
  if (V->n > (int64_t(1) << 20)) throw Error(TAMM_EUNSUPPORTED, "triples: virtual space too large");
}

std::string triples_key(const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vo, const tamm_tensor* Vv,
                        const tamm_tensor* Voo, int64_t ws) {
  return "triples|" + std::to_string(T2->id) + "|" + std::to_string(T1->id) + "|" + std::to_string(Vo->id) + "|" +
         std::to_string(Vv->id) + "|" + std::to_string(Voo->id) + "|" + std::to_string(ws);
}

}  // namespace

void triples_info(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vo,
                  const tamm_tensor* Vv, const tamm_tensor* Voo, int64_t workspace_bytes, int64_t* n_triples,
                  double* gemm_flops, int* n_batches) {
  check_triples_inputs(T2, T1, Vo, Vv, Voo);
  TriplesPlan p(ctx, *T2, *T1, *Vo, *Vv, *Voo, workspace_bytes, false);
  if (n_triples) *n_triples = (int64_t)p.triples.size();
  if (gemm_flops) *gemm_flops = p.gemm_flops;
  if (n_batches) *n_batches = (int)p.n_batches;
}

void run_triples(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1, const tamm_tensor* Vo,
                 const tamm_tensor* Vv, const tamm_tensor* Voo, const double* eps_o, const double* eps_v,
                 int precision, int slices, int64_t workspace_bytes, double* energy, double* triple_energies) {
  check_triples_inputs(T2, T1, Vo, Vv, Voo);
  if (!eps_o || !eps_v || !energy) throw Error(TAMM_EINVAL, "triples: null device pointer");
  for (const tamm_tensor* X : {T2, T1, Vo, Vv, Voo})
    if (X->n_elems && !X->data) throw Error(TAMM_EINVAL, "triples: tensor has no storage");
  if (precision != TAMM_PREC_F64 && precision != TAMM_PREC_OZAKI_BF16)
    throw Error(TAMM_EUNSUPPORTED, "triples: precision must be TAMM_PREC_F64 or TAMM_PREC_OZAKI_BF16");
  if (precision == TAMM_PREC_OZAKI_BF16) {
    if (slices == 0) slices = kOzDefaultSlices;
    if (slices < kOzMinSlices || slices > kOzMaxSlices) throw Error(TAMM_EINVAL, "triples: slices must be 3..8");
  }
  if (ctx->group_active) throw Error(TAMM_EINVAL, "triples: not inside a contraction group");
  const std::string key = triples_key(T2, T1, Vo, Vv, Voo, workspace_bytes);
  TriplesPlan* p;
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    p = static_cast<TriplesPlan*>(it->second.get());
  } else {
    if (ctx->capturing) throw Error(TAMM_EINVAL, "a new triples plan cannot be built during graph capture");
    p = new TriplesPlan(ctx, *T2, *T1, *Vo, *Vv, *Voo, workspace_bytes, true);
    p->t2_ = T2;
    p->vo_ = Vo;
    p->vv_ = Vv;
    ctx->plans[key].reset(p);
  }
  if (precision == TAMM_PREC_OZAKI_BF16) {
    if (ctx->capturing && (p->oz_S != slices || p->oz_policy != ctx->oz_tile_policy || p->oz_shared != ctx->oz_shared))
      throw Error(TAMM_EINVAL, "triples: split-precision images must be planned before graph capture");
    p->build_split(slices, ctx->oz_tile_policy, ctx->oz_shared);
  }
  // scratch: U workspace, partials, then (split path) images and exponents
  auto align = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  const size_t ws_bytes = align((size_t)std::max<int64_t>(p->ws_elems, 1) * 8);
  const size_t part_bytes = align((size_t)std::max<int64_t>(p->n_eitems, 1) * kEnergyWarps * 8);
  size_t total = ws_bytes + part_bytes;
  // double-float copies of V_oovv, T1 and the orbital energies (8 bytes per element each)
  const size_t off_dv = total;
  total += align((size_t)std::max<int64_t>(Voo->n_elems, 1) * 8);
  const size_t off_dt = total;
  total += align((size_t)std::max<int64_t>(T1->n_elems, 1) * 8);
  const size_t off_deo = total;
  total += align((size_t)std::max<int64_t>(p->no, 1) * 8);
  const size_t off_dev = total;
  total += align((size_t)std::max<int64_t>(p->nv, 1) * 8);
  size_t off_a = 0, off_b = 0, off_ea = 0, off_eb = 0, off_sa = 0, off_sb = 0;
  if (precision == TAMM_PREC_OZAKI_BF16) {
    if (p->oz_shared) {
      off_sa = total;
      total += align((size_t)std::max<int64_t>(p->slots_a, 1) * 8);
      off_sb = total;
      total += align((size_t)std::max<int64_t>(p->slots_b, 1) * 8);
    }
    off_a = total;
    total += align((size_t)p->a_bytes);
    off_b = total;
    total += align((size_t)p->b_bytes);
    off_ea = total;
    total += align((size_t)p->a_rows * 4);
    off_eb = total;
    total += align((size_t)p->b_rows * 4);
  }
  char* scratch = (char*)ctx_scratch(ctx, total);
  double* U = (double*)scratch;
  double* partials = (double*)(scratch + ws_bytes);
  float2* dvoo = (float2*)(scratch + off_dv);
  float2* dt1 = (float2*)(scratch + off_dt);
  float2* deo = (float2*)(scratch + off_deo);
  float2* dev = (float2*)(scratch + off_dev);
  cuda_check(launch_to_df(ctx, Voo->data, Voo->n_elems, dvoo), "triples double-float copy");
  cuda_check(launch_to_df(ctx, T1->data, T1->n_elems, dt1), "triples double-float copy");
  cuda_check(launch_to_df(ctx, eps_o, p->no, deo), "triples double-float copy");
  cuda_check(launch_to_df(ctx, eps_v, p->nv, dev), "triples double-float copy");
  // GEMM-order copies of the inputs
  const double one = 1.0;
  p->copy_q->run(p->Tq->data, T2->data, 0.0, &one);
  p->copy_p->run(p->Vp->data, Vv->data, 0.0, &one);
  p->copy_z->run(p->Tz->data, T2->data, 0.0, &one);
  uint8_t *ta = nullptr, *tb = nullptr;
  int32_t *ea = nullptr, *eb = nullptr;
  if (precision == TAMM_PREC_OZAKI_BF16) {
    ta = (uint8_t*)(scratch + off_a);
    tb = (uint8_t*)(scratch + off_b);
    ea = (int32_t*)(scratch + off_ea);
    eb = (int32_t*)(scratch + off_eb);
    const double* src[4] = {p->Tq->data, p->Vp->data, Vo->data, p->Tz->data};
    if (p->oz_shared) {
      // one exponent per U row and column over all six block pairs: maxima first, then the slices
      unsigned long long* sm[2] = {(unsigned long long*)(scratch + off_sa), (unsigned long long*)(scratch + off_sb)};
      cuda_check(cudaMemsetAsync(sm[0], 0, (size_t)p->slots_a * 8, ctx->stream), "triples maxima clear");
      cuda_check(cudaMemsetAsync(sm[1], 0, (size_t)p->slots_b * 8, ctx->stream), "triples maxima clear");
      for (int mode : {kOzSliceSharedMax, kOzSliceSharedPack})
        for (int s = 0; s < 4; ++s)
          cuda_check(launch_ozaki_slice(ctx, src[s], p->d_rec[s], p->d_sitems[s], (int64_t)p->sitems[s].size(),
                                        slices, false, s < 2 ? ta : tb, s < 2 ? ea : eb, p->warps[s], p->kbuf[s],
                                        mode, sm[s < 2 ? 0 : 1]),
                     "triples slicing");
    } else {
      for (int s = 0; s < 4; ++s)
        cuda_check(launch_ozaki_slice(ctx, src[s], p->d_rec[s], p->d_sitems[s], (int64_t)p->sitems[s].size(), slices,
                                      false, s < 2 ? ta : tb, s < 2 ? ea : eb, p->warps[s], p->kbuf[s]),
                   "triples slicing");
    }
  }
  for (int64_t bch = 0; bch < p->n_batches; ++bch) {
    if (precision == TAMM_PREC_F64) {
      const int64_t i0 = p->fitem_begin[(size_t)bch], i1 = p->fitem_begin[(size_t)bch + 1];
      cuda_check(launch_gemm_f64(ctx, p->Tq->data, Vo->data, U, p->d_fgroups_q, p->d_ftasks_q, p->d_fitems + i0,
                                 i1 - i0, 1.0, 0.0),
                 "triples gemm (occupied sums)");
      cuda_check(launch_gemm_f64(ctx, p->Vp->data, p->Tz->data, U, p->d_fgroups_z, p->d_ftasks_z, p->d_fitems + i0,
                                 i1 - i0, 1.0, 1.0),
                 "triples gemm (virtual sums)");
    } else {
      const int64_t i0 = p->oitem_begin[(size_t)bch], i1 = p->oitem_begin[(size_t)bch + 1];
      OzProblem pr;
      memset(&pr, 0, sizeof(pr));
      pr.a_tiles = ta;
      pr.b_tiles = tb;
      pr.a_exp = ea;
      pr.b_exp = eb;
      pr.groups = p->d_ogroups;
      pr.tasks = p->d_otasks;
      pr.items = p->d_oitems + i0;
      pr.c = U;
      pr.alpha = 1.0;
      pr.beta = 0.0;
      pr.alpha_pow2 = 1;
      pr.alpha_exp = 0;
      int64_t n = i1 - i0;
      cuda_check(launch_ozaki_gemm(ctx, &pr, &n, 1, slices, ctx->oz_chunk_k / kOzTileK, ctx->oz_persistent),
                 "triples gemm (split precision)");
    }
    const int64_t e0 = p->eitem_begin[(size_t)bch], e1 = p->eitem_begin[(size_t)bch + 1];
    cuda_check(launch_triples_energy(ctx, U, p->d_eitems + e0, e1 - e0, dvoo, dt1, deo, dev,
                                     partials + e0 * kEnergyWarps),
               "triples energy");
  }
  cuda_check(launch_reduce_final(ctx, partials, p->n_eitems * kEnergyWarps, 1.0, 0, energy), "triples reduction");
  if (triple_energies && !p->triples.empty())
    cuda_check(launch_triples_segments(ctx, partials, p->d_seg, (int64_t)p->triples.size(), triple_energies),
               "triples per-triple sums");
}

cudaError_t launch_to_df(tamm_ctx* ctx, const double* x, int64_t n, float2* out) {
  if (n == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_TRIPLES);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8L * std::max(1, ctx->sm_count));
  to_df_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(x, n, out);
  kernel_end(ctx, TAMM_KERNEL_TRIPLES);
  return cudaGetLastError();
}

cudaError_t launch_triples_energy(tamm_ctx* ctx, const double* U, const void* items, int64_t n_items,
                                  const float2* voo, const float2* t1, const float2* eps_o, const float2* eps_v,
                                  double* partials) {
  if (n_items == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_TRIPLES);
  triples_energy_kernel<<<(unsigned)n_items, 32 * kEnergyWarps, 0, ctx->stream>>>(U, (const TriplesItem*)items, voo,
                                                                                  t1, eps_o, eps_v, partials);
  kernel_end(ctx, TAMM_KERNEL_TRIPLES);
  return cudaGetLastError();
}

cudaError_t launch_triples_segments(tamm_ctx* ctx, const double* partials, const int64_t* seg, int64_t n,
                                    double* out) {
  if (n == 0) return cudaSuccess;
  kernel_begin(ctx, TAMM_KERNEL_REDUCE);
  triples_segment_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(partials, seg, n, out);
  kernel_end(ctx, TAMM_KERNEL_REDUCE);
  return cudaGetLastError();
}

}  // namespace tamm
