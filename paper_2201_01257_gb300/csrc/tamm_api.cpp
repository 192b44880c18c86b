// C ABI of the block-sparse contraction library: contexts, tiled index spaces,
// block-sparse tensors, and the host planner that turns a labelled operation
// into device task lists (Sec. III.A operations; Sec. III.B sparsity-aware
// block storage).  All device work is enqueued on the context's stream.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>

#include "tamm_internal.h"
#include "tamm_contract.h"
#include "tamm_lambda.h"
#include "tamm_plan.h"
#include "tamm_triples.h"

using namespace tamm;

// ------------------------------------------------------------------ errors

namespace tamm {

Error::Error(tamm_status s, const char* fmt, ...) : status(s) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  msg = buf;
}

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw Error(TAMM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace tamm

template <class F>
static tamm_status guarded(tamm_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->last_error.clear();
    return TAMM_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    if (ctx && ctx->capturing) ctx->capture_failed = true;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    if (ctx && ctx->capturing) ctx->capture_failed = true;
    return TAMM_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what();
    if (ctx && ctx->capturing) ctx->capture_failed = true;
    return TAMM_EINVAL;
  }
}

// Operations other than split-precision contractions run at once, so inside a
// group they would overtake the recorded contractions: refuse them.
static void no_group(tamm_ctx* ctx, const char* what) {
  if (ctx->group_active) throw Error(TAMM_EINVAL, "%s cannot be issued inside a contraction group", what);
}

// --------------------------------------------------------------- allocation

namespace tamm {

void require_device(tamm_ctx* ctx) {
  if (ctx->host_only) throw Error(TAMM_ECUDA, "host-only context (device -1) cannot run device work");
}

void* ctx_alloc(tamm_ctx* ctx, size_t bytes) {
  require_device(ctx);
  if (ctx->capturing)
    throw Error(TAMM_EINVAL, "device allocation of %zu bytes during graph capture (run the same operations once "
                "before capturing so that plans and scratch exist)", bytes);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (ctx->allocator.alloc) {
    p = ctx->allocator.alloc(bytes, (void*)ctx->stream, ctx->allocator.user);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) throw Error(TAMM_ENOMEM, "device allocation of %zu bytes failed", bytes);
  return p;
}

void ctx_free(tamm_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  if (ctx->allocator.release) {
    ctx->allocator.release(p, bytes, (void*)ctx->stream, ctx->allocator.user);
  } else {
    cudaFreeAsync(p, ctx->stream);
  }
}

void* ctx_scratch(tamm_ctx* ctx, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->scratch.bytes < bytes) {
    if (ctx->capturing) throw Error(TAMM_EINVAL, "scratch growth during graph capture");
    const size_t grow = std::max(bytes, ctx->scratch.bytes + ctx->scratch.bytes / 4);
    ctx_free(ctx, ctx->scratch.ptr, ctx->scratch.bytes);
    ctx->scratch.ptr = nullptr;
    ctx->scratch.bytes = 0;
    ctx->scratch.ptr = ctx_alloc(ctx, grow);
    ctx->scratch.bytes = grow;
  }
  return ctx->scratch.ptr;
}

double* ctx_reduce_buffer(tamm_ctx* ctx, size_t n) {
  if (ctx->reduce_cap < n) {
    if (ctx->capturing) throw Error(TAMM_EINVAL, "reduction buffer growth during graph capture");
    ctx_free(ctx, ctx->d_reduce, ctx->reduce_cap * sizeof(double));
    ctx->d_reduce = nullptr;
    ctx->reduce_cap = 0;
    ctx->d_reduce = (double*)ctx_alloc(ctx, n * sizeof(double));
    ctx->reduce_cap = n;
  }
  return ctx->d_reduce;
}

Plan::~Plan() {
  for (auto& b : bufs) ctx_free(ctx, b.ptr, b.bytes);
}

void* Plan::upload_bytes(const void* host, size_t bytes) {
  void* d = ctx_alloc(ctx, bytes);
  bufs.push_back({d, bytes});
  if (bytes) cuda_check(cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, ctx->stream), "plan upload");
  return d;
}

}  // namespace tamm

// ---------------------------------------------------------------- context

extern "C" tamm_status tamm_ctx_create(int device, void* stream, tamm_alloc_fn alloc, tamm_free_fn release,
                                       void* user, tamm_ctx** out) {
  if (!out) return TAMM_EINVAL;
  *out = nullptr;
  if ((alloc == nullptr) != (release == nullptr)) return TAMM_EINVAL;
  tamm_ctx* ctx = new (std::nothrow) tamm_ctx();
  if (!ctx) return TAMM_ENOMEM;
  tamm_status st = guarded(ctx, [&] {
    ctx->device = device;
    if (device < 0) {  // host-only context: metadata, plans and flop counts, no device work
      ctx->host_only = true;
      return;
    }
    cuda_check(cudaSetDevice(device), "cudaSetDevice");
    ctx->stream = (cudaStream_t)stream;
    ctx->allocator = {alloc, release, user};
    cuda_check(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device), "attribute");
    ctx->d_status = (int*)ctx_alloc(ctx, 256);
    cuda_check(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream), "memset status");
    cuda_check(cudaMallocHost(&ctx->h_result, 64), "cudaMallocHost");
  });
  if (st != TAMM_OK) {
    tamm_ctx_destroy(ctx);
    return st;
  }
  *out = ctx;
  return TAMM_OK;
}

extern "C" tamm_status tamm_ctx_set_stream(tamm_ctx* ctx, void* stream) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (ctx->capturing || ctx->group_active) throw Error(TAMM_EINVAL, "stream change inside a group or capture");
    cuda_check(cudaStreamSynchronize(ctx->stream), "stream sync");
    ctx->stream = (cudaStream_t)stream;
  });
}

extern "C" void tamm_ctx_destroy(tamm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->host_only) {
    delete ctx;
    return;
  }
  cudaSetDevice(ctx->device);
  for (auto& d : ctx->deferred_graphs) {
    if (d.second) cudaGraphExecDestroy(d.second);
    if (d.first) cudaGraphDestroy(d.first);
  }
  ctx->deferred_graphs.clear();
  ctx->plans.clear();
  ctx_free(ctx, ctx->scratch.ptr, ctx->scratch.bytes);
  ctx_free(ctx, ctx->d_reduce, ctx->reduce_cap * sizeof(double));
  ctx_free(ctx, ctx->d_status, 256);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->h_result) cudaFreeHost(ctx->h_result);
  for (auto& t : ctx->timed) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  (void)cudaGetLastError();
  delete ctx;
}

extern "C" tamm_status tamm_ctx_set_option(tamm_ctx* ctx, int option, int64_t value) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    if (option == TAMM_OPT_OZAKI_CHUNK_K) {
      if (value < 16 || value > 1280 || value % 16) throw Error(TAMM_EINVAL, "chunk must be a multiple of 16 in 16..1280");
      ctx->oz_chunk_k = (int)value;
      return;
    }
    if (option == TAMM_OPT_OZAKI_TILE_POLICY) {
      if (value < 0 || value > 3) throw Error(TAMM_EINVAL, "tile policy must be 0..3");
      ctx->oz_tile_policy = (int)value;
      return;
    }
    if (option == TAMM_OPT_OZAKI_SPLIT_K) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "split must be 0 or 1");
      ctx->oz_split = value != 0;
      return;
    }
    if (option == TAMM_OPT_OZAKI_PANELS) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "panels must be 0 or 1");
      ctx->oz_panels = value != 0;
      return;
    }
    if (option == TAMM_OPT_OZAKI_PERSISTENT) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "persistent must be 0 or 1");
      ctx->oz_persistent = value != 0;
      return;
    }
    if (option == TAMM_OPT_OZAKI_SHARED_SCALE) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "shared scale must be 0 or 1");
      ctx->oz_shared = value != 0;
      return;
    }
    if (option == TAMM_OPT_OZAKI_FUSED_A) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "fused A must be 0 or 1");
      ctx->oz_fused_a = value != 0;
      return;
    }
    if (option == TAMM_OPT_WAIT_CYCLES) {
      if (value < 1000) throw Error(TAMM_EINVAL, "wait limit must be at least 1000 cycles");
      ctx->oz_wait_cycles = (long long)value;
      return;
    }
    if (option == TAMM_OPT_TEST_WITHHOLD_COPY) {
      if (value != 0 && value != 1) throw Error(TAMM_EINVAL, "withhold must be 0 or 1");
      ctx->oz_test_withhold = (int)value;
      return;
    }
    throw Error(TAMM_EINVAL, "unknown option %d", option);
  });
}

extern "C" const char* tamm_last_error(const tamm_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

namespace tamm {
// Synchronise and turn a recorded device status into an error.
void sync_and_check(tamm_ctx* ctx) {
  if (ctx->capturing) throw Error(TAMM_EINVAL, "synchronising call during graph capture");
  cuda_check(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  int st = 0;
  cuda_check(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (st != 0) {
    cuda_check(cudaMemset(ctx->d_status, 0, sizeof(int)), "status clear");
    if (st == TAMM_ETIMEOUT) throw Error(TAMM_ETIMEOUT, "a bounded device-side wait ran out");
    throw Error(st, "device-side check failed (status %d)", st);
  }
}
}  // namespace tamm

extern "C" tamm_status tamm_sync(tamm_ctx* ctx) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    sync_and_check(ctx);
  });
}

// ----------------------------------------------------------------- spaces

extern "C" tamm_status tamm_space_create(tamm_ctx* ctx, int n_groups, const int64_t* group_size,
                                         const int* group_spin, const int* group_irrep, int n_tiles,
                                         const int64_t* tile_sizes, int64_t fixed_tile, tamm_space** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    if (n_groups <= 0 || !group_size || !group_spin) throw Error(TAMM_EINVAL, "space: need at least one group");
    if (fixed_tile <= 0 && (n_tiles <= 0 || !tile_sizes))
      throw Error(TAMM_EINVAL, "space: give a fixed tile size or an explicit tile list");
    std::unique_ptr<tamm_space> s(new tamm_space());
    s->ctx = ctx;
    s->id = ctx->next_id++;
    int t = 0;
    int64_t pos = 0;
    for (int g = 0; g < n_groups; ++g) {
      if (group_size[g] < 0) throw Error(TAMM_EINVAL, "space: negative group size");
      if (group_spin[g] < -1 || group_spin[g] > 1) throw Error(TAMM_EINVAL, "space: spin must be +1, -1 or 0");
      const int irr = group_irrep ? group_irrep[g] : 0;
      if (irr < 0 || irr > 7) throw Error(TAMM_EINVAL, "space: irrep must be in 0..7");
      int64_t left = group_size[g];
      while (left > 0) {
        int64_t ts;
        if (fixed_tile > 0) {
          ts = std::min(left, fixed_tile);
        } else {
          if (t >= n_tiles) throw Error(TAMM_EINVAL, "space: tile list does not cover group %d", g);
          ts = tile_sizes[t];
          if (ts <= 0 || ts > left) throw Error(TAMM_EINVAL, "space: tile %d straddles group %d", t, g);
        }
        s->off.push_back(pos);
        s->size.push_back(ts);
        s->spin.push_back(group_spin[g]);
        s->irrep.push_back(irr);
        pos += ts;
        left -= ts;
        ++t;
      }
    }
    if (fixed_tile <= 0 && t != n_tiles) throw Error(TAMM_EINVAL, "space: %d tile sizes given, %d used", n_tiles, t);
    if (t == 0) throw Error(TAMM_EINVAL, "space: empty");
    s->n_tiles = t;
    s->n = pos;
    *out = s.release();
  });
}

extern "C" tamm_status tamm_space_info(const tamm_space* s, int* n_tiles, int64_t* n) {
  if (!s) return TAMM_EINVAL;
  if (n_tiles) *n_tiles = s->n_tiles;
  if (n) *n = s->n;
  return TAMM_OK;
}

extern "C" tamm_status tamm_space_tiles(const tamm_space* s, int64_t* offset, int64_t* size, int* spin,
                                        int* irrep) {
  if (!s) return TAMM_EINVAL;
  for (int t = 0; t < s->n_tiles; ++t) {
    if (offset) offset[t] = s->off[t];
    if (size) size[t] = s->size[t];
    if (spin) spin[t] = s->spin[t];
    if (irrep) irrep[t] = s->irrep[t];
  }
  return TAMM_OK;
}

extern "C" void tamm_space_destroy(tamm_space* s) { delete s; }

// ---------------------------------------------------------------- tensors

namespace tamm {

static bool block_rule(const tamm_tensor& T, const int64_t* tt) {
  if (T.sym == TAMM_SYM_DENSE) return true;
  int up = 0, lo = 0, x = 0;
  for (int m = 0; m < T.nm; ++m) {
    const int s = T.sp[m]->spin[(size_t)tt[m]];
    (m < T.n_upper ? up : lo) += s;
    x ^= T.sp[m]->irrep[(size_t)tt[m]];
  }
  if (up != lo) return false;
  if (T.sym == TAMM_SYM_SPIN_IRREP && x != 0) return false;
  return true;
}

// Fill lookup/tiles/off from a predicate on tile tuples (lexicographic order).
template <class Pred>
static void build_blocks(tamm_tensor& T, Pred keep) {
  int64_t n_tuples = 1;
  for (int m = 0; m < T.nm; ++m) {
    n_tuples *= T.sp[m]->n_tiles;
    if (n_tuples > (int64_t(1) << 31)) throw Error(TAMM_EINVAL, "tensor: too many tile tuples");
  }
  T.lookup.assign((size_t)n_tuples, -1);
  T.tiles.clear();
  T.off.assign(1, 0);
  int64_t tt[kMaxModes];
  int64_t pos = 0, nb = 0;
  for (int64_t lin = 0; lin < n_tuples; ++lin) {
    int64_t r = lin;
    for (int m = T.nm - 1; m >= 0; --m) {
      tt[m] = r % T.sp[m]->n_tiles;
      r /= T.sp[m]->n_tiles;
    }
    if (!keep(tt)) continue;
    int64_t sz = 1;
    for (int m = 0; m < T.nm; ++m) {
      T.tiles.push_back(tt[m]);
      sz *= T.sp[m]->size[(size_t)tt[m]];
    }
    T.lookup[(size_t)lin] = nb++;
    pos += sz;
    T.off.push_back(pos);
  }
  T.n_blocks = nb;
  T.n_elems = pos;
}

void build_blocks_where(tamm_tensor& T, const std::function<bool(const int64_t*)>& keep) { build_blocks(T, keep); }

static void not_lambda(const tamm_tensor* t, const char* what) {
  if (t->lambda) throw Error(TAMM_EUNSUPPORTED, "%s: a lambda tensor has no storage", what);
}

std::unique_ptr<tamm_tensor> make_permuted_tensor(const tamm_tensor& S, const int* perm) {
  // New tensor whose mode m is S's mode perm[m]; stores exactly the images of S's blocks.
  std::unique_ptr<tamm_tensor> T(new tamm_tensor());
  T->ctx = S.ctx;
  T->id = S.ctx->next_id++;
  T->nm = S.nm;
  T->n_upper = -1;
  T->sym = -1;
  for (int m = 0; m < S.nm; ++m) T->sp[m] = S.sp[perm[m]];
  build_blocks(*T, [&](const int64_t* tt) {
    int64_t st[kMaxModes];
    for (int m = 0; m < S.nm; ++m) st[perm[m]] = tt[m];
    return S.find(st) >= 0;
  });
  return T;
}

}  // namespace tamm

extern "C" tamm_status tamm_tensor_create(tamm_ctx* ctx, int n_modes, tamm_space* const* modes, int n_upper,
                                          int symmetry, tamm_tensor** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    if (n_modes <= 0 || n_modes > kMaxModes || !modes) throw Error(TAMM_EINVAL, "tensor: 1..8 modes");
    if (n_upper < 0 || n_upper > n_modes) throw Error(TAMM_EINVAL, "tensor: n_upper out of range");
    if (symmetry < TAMM_SYM_DENSE || symmetry > TAMM_SYM_SPIN_IRREP) throw Error(TAMM_EINVAL, "tensor: symmetry");
    std::unique_ptr<tamm_tensor> T(new tamm_tensor());
    T->ctx = ctx;
    T->id = ctx->next_id++;
    T->nm = n_modes;
    T->n_upper = n_upper;
    T->sym = symmetry;
    for (int m = 0; m < n_modes; ++m) {
      if (!modes[m]) throw Error(TAMM_EINVAL, "tensor: null space");
      T->sp[m] = modes[m];
    }
    build_blocks(*T, [&](const int64_t* tt) { return block_rule(*T, tt); });
    *out = T.release();
  });
}

extern "C" tamm_status tamm_tensor_create_permuted(tamm_ctx* ctx, const tamm_tensor* like, const int* perm,
                                                   tamm_tensor** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    if (!like || !perm) throw Error(TAMM_EINVAL, "permuted tensor: null argument");
    bool seen[kMaxModes] = {};
    for (int m = 0; m < like->nm; ++m) {
      if (perm[m] < 0 || perm[m] >= like->nm || seen[perm[m]]) throw Error(TAMM_EINVAL, "permuted tensor: bad perm");
      seen[perm[m]] = true;
    }
    *out = make_permuted_tensor(*like, perm).release();
  });
}

extern "C" tamm_status tamm_tensor_info(const tamm_tensor* t, int64_t* n_blocks, int64_t* n_elems) {
  if (!t) return TAMM_EINVAL;
  if (n_blocks) *n_blocks = t->n_blocks;
  if (n_elems) *n_elems = t->n_elems;
  return TAMM_OK;
}

extern "C" tamm_status tamm_tensor_blocks(const tamm_tensor* t, int64_t* block_tiles, int64_t* block_offsets) {
  if (!t) return TAMM_EINVAL;
  if (block_tiles && !t->tiles.empty()) memcpy(block_tiles, t->tiles.data(), t->tiles.size() * sizeof(int64_t));
  if (block_offsets && t->n_blocks) memcpy(block_offsets, t->off.data(), (size_t)t->n_blocks * sizeof(int64_t));
  return TAMM_OK;
}

extern "C" tamm_status tamm_tensor_bind(tamm_tensor* t, double* device_data) {
  if (!t) return TAMM_EINVAL;
  return guarded(t->ctx, [&] {
    require_device(t->ctx);
    not_lambda(t, "bind");
    if (!device_data && t->n_elems) throw Error(TAMM_EINVAL, "bind: null device pointer");
    if (((uintptr_t)device_data) % 8) throw Error(TAMM_EINVAL, "bind: pointer not 8-byte aligned");
    if (t->owned) ctx_free(t->ctx, t->data, t->owned_bytes);
    t->owned = false;
    t->owned_bytes = 0;
    t->data = device_data;
  });
}

extern "C" tamm_status tamm_tensor_allocate(tamm_tensor* t) {
  if (!t) return TAMM_EINVAL;
  return guarded(t->ctx, [&] {
    not_lambda(t, "allocate");
    if (t->owned) ctx_free(t->ctx, t->data, t->owned_bytes);
    t->owned = false;
    const size_t bytes = (size_t)std::max<int64_t>(t->n_elems, 1) * sizeof(double);
    t->data = (double*)ctx_alloc(t->ctx, bytes);
    t->owned = true;
    t->owned_bytes = bytes;
  });
}

extern "C" tamm_status tamm_tensor_copy_from_host(tamm_ctx* ctx, tamm_tensor* t, const double* host) {
  if (!ctx || !t) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    not_lambda(t, "copy");
    if (!host || (t->n_elems && !t->data)) throw Error(TAMM_EINVAL, "copy: null buffer or unbound tensor");
    cuda_check(cudaMemcpyAsync(t->data, host, (size_t)t->n_elems * sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream),
               "host to device copy");
  });
}

extern "C" tamm_status tamm_tensor_copy_to_host(tamm_ctx* ctx, const tamm_tensor* t, double* host) {
  if (!ctx || !t) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    not_lambda(t, "copy");
    if (!host || (t->n_elems && !t->data)) throw Error(TAMM_EINVAL, "copy: null buffer or unbound tensor");
    cuda_check(cudaMemcpyAsync(host, t->data, (size_t)t->n_elems * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream),
               "device to host copy");
  });
}

extern "C" double* tamm_tensor_data(const tamm_tensor* t) { return t ? t->data : nullptr; }

extern "C" tamm_status tamm_tensor_create_cholesky(tamm_ctx* ctx, const tamm_tensor* X, int64_t slab_bytes,
                                                   tamm_tensor** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] { *out = make_cholesky_tensor(ctx, X, slab_bytes).release(); });
}

extern "C" tamm_status tamm_cholesky_info(const tamm_tensor* V, int* n_slabs, double* form_flops,
                                          int64_t* buffer_bytes) {
  if (!V || !V->lambda) return TAMM_EINVAL;
  if (n_slabs) *n_slabs = (int)V->lambda->slabs.size();
  if (form_flops) *form_flops = V->lambda->form_flops;
  if (buffer_bytes) *buffer_bytes = (int64_t)(V->lambda->v_bytes + V->lambda->x1_bytes);
  return TAMM_OK;
}

extern "C" tamm_status tamm_cholesky_form(tamm_ctx* ctx, const tamm_tensor* V, tamm_tensor* out, int precision,
                                          int slices) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    cholesky_form(ctx, V, out, precision, slices);
  });
}

extern "C" void tamm_tensor_destroy(tamm_tensor* t) {
  if (!t) return;
  if (t->owned) ctx_free(t->ctx, t->data, t->owned_bytes);
  delete t;
}

// ------------------------------------------------------------- operations

extern "C" tamm_status tamm_contract(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                                     const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb,
                                     int precision, int slices) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (ctx->group_active && precision != TAMM_PREC_OZAKI_BF16 && precision != TAMM_PREC_BF16X3)
      throw Error(TAMM_EINVAL, "only split-precision contractions can be grouped");
    run_contract(ctx, alpha, C, lc, beta, A, la, B, lb, precision, slices);
  });
}

extern "C" tamm_status tamm_contract_flops(tamm_ctx* ctx, const tamm_tensor* C, const char* lc,
                                           const tamm_tensor* A, const char* la, const tamm_tensor* B,
                                           const char* lb, double* flops) {
  if (!ctx || !flops) return TAMM_EINVAL;
  return guarded(ctx, [&] { *flops = contract_flops(ctx, C, lc, A, la, B, lb); });
}

extern "C" tamm_status tamm_add(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A,
                                int n_terms, const char* const* la, const double* alpha) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    no_group(ctx, "an add");
    run_add(ctx, C, lc, beta, A, n_terms, la, alpha);
  });
}

extern "C" tamm_status tamm_add_scaled(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta,
                                       const tamm_tensor* A, int n_terms, const char* const* la, const double* alpha,
                                       const double* scale_device) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    no_group(ctx, "an add");
    if (!scale_device) throw Error(TAMM_EINVAL, "add: null scale pointer");
    if (((uintptr_t)scale_device) % 8) throw Error(TAMM_EINVAL, "add: scale pointer not 8-byte aligned");
    run_add(ctx, C, lc, beta, A, n_terms, la, alpha, scale_device);
  });
}

namespace {
// dX must have X's spaces and block table, so that its packed layout is X's.
void same_blocks(const tamm_tensor* X, const tamm_tensor* dX, const char* what) {
  if (dX->nm != X->nm) throw Error(TAMM_EINVAL, "adjoint: %s has %d modes, its operand %d", what, dX->nm, X->nm);
  for (int m = 0; m < X->nm; ++m)
    if (dX->sp[m] != X->sp[m]) throw Error(TAMM_EINVAL, "adjoint: %s mode %d is on another space", what, m);
  if (dX->n_blocks != X->n_blocks || dX->tiles != X->tiles)
    throw Error(TAMM_EINVAL, "adjoint: %s stores other blocks than its operand", what);
}
}  // namespace

extern "C" tamm_status tamm_contract_adjoint(tamm_ctx* ctx, double alpha, const tamm_tensor* dC, const char* lc,
                                             const tamm_tensor* A, const char* la, const tamm_tensor* B,
                                             const char* lb, tamm_tensor* dA, tamm_tensor* dB, double beta,
                                             int precision, int slices) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!dC || !A || !B || !lc || !la || !lb) throw Error(TAMM_EINVAL, "adjoint: null argument");
    if (!dA && !dB) throw Error(TAMM_EINVAL, "adjoint: neither dA nor dB requested");
    if (ctx->group_active && precision != TAMM_PREC_OZAKI_BF16 && precision != TAMM_PREC_BF16X3)
      throw Error(TAMM_EINVAL, "only split-precision contractions can be grouped");
    // the forward contraction itself must be valid: its label analysis rejects what it would
    (void)contract_flops(ctx, dC, lc, A, la, B, lb);
    if (dA) same_blocks(A, dA, "dA");
    if (dB) same_blocks(B, dB, "dB");
    if (dA && dB && dA->data && dA->data == dB->data) throw Error(TAMM_EINVAL, "adjoint: dA and dB alias");
    // the adjoint of a MultOp is a MultOp with the label roles exchanged
    if (dA) run_contract(ctx, alpha, dA, la, beta, dC, lc, B, lb, precision, slices);
    if (dB) run_contract(ctx, alpha, dB, lb, beta, A, la, dC, lc, precision, slices);
  });
}

extern "C" tamm_status tamm_triples_energy(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1,
                                           const tamm_tensor* Vooov, const tamm_tensor* Vvovv,
                                           const tamm_tensor* Voovv, const double* eps_occ, const double* eps_virt,
                                           int precision, int slices, int64_t workspace_bytes,
                                           double* energy_device, double* triple_energies_device) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    no_group(ctx, "a triples correction");
    run_triples(ctx, T2, T1, Vooov, Vvovv, Voovv, eps_occ, eps_virt, precision, slices, workspace_bytes,
                energy_device, triple_energies_device);
  });
}

extern "C" tamm_status tamm_triples_info(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1,
                                         const tamm_tensor* Vooov, const tamm_tensor* Vvovv, const tamm_tensor* Voovv,
                                         int64_t workspace_bytes, int64_t* n_triples, double* gemm_flops,
                                         int* n_batches) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    triples_info(ctx, T2, T1, Vooov, Vvovv, Voovv, workspace_bytes, n_triples, gemm_flops, n_batches);
  });
}

extern "C" tamm_status tamm_energy_async(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la,
                                         const tamm_tensor* B, const char* lb, double* result_device) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!result_device) throw Error(TAMM_EINVAL, "energy: null result pointer");
    no_group(ctx, "an energy");
    run_energy(ctx, alpha, A, la, B, lb, result_device);
  });
}

extern "C" tamm_status tamm_energy(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la,
                                   const tamm_tensor* B, const char* lb, double* result_host) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!result_host) throw Error(TAMM_EINVAL, "energy: null result pointer");
    no_group(ctx, "an energy");
    if (ctx->capturing) throw Error(TAMM_EINVAL, "synchronising call during graph capture");
    double* out = result_slot(ctx, 0);
    run_energy(ctx, alpha, A, la, B, lb, out);
    cuda_check(cudaMemcpyAsync(ctx->h_result, out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    sync_and_check(ctx);
    *result_host = ctx->h_result[0];
  });
}

extern "C" tamm_status tamm_norm_async(tamm_ctx* ctx, const tamm_tensor* t, double* result_device) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!result_device) throw Error(TAMM_EINVAL, "norm: null result pointer");
    no_group(ctx, "a norm");
    run_norm(ctx, t, result_device);
  });
}

extern "C" tamm_status tamm_norm(tamm_ctx* ctx, const tamm_tensor* t, double* result_host) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!result_host) throw Error(TAMM_EINVAL, "norm: null result pointer");
    no_group(ctx, "a norm");
    if (ctx->capturing) throw Error(TAMM_EINVAL, "synchronising call during graph capture");
    double* out = result_slot(ctx, 1);
    run_norm(ctx, t, out);
    cuda_check(cudaMemcpyAsync(ctx->h_result, out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    sync_and_check(ctx);
    *result_host = ctx->h_result[0];
  });
}

// ------------------------------------------------- groups and graph capture

namespace {

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || !na || !nb) return false;
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

}  // namespace

struct tamm_graph {
  tamm_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;  // kernels one replay runs
};

extern "C" tamm_status tamm_group_begin(tamm_ctx* ctx) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (ctx->group_active) throw Error(TAMM_EINVAL, "a contraction group is already open");
    ctx->group_active = true;
    ctx->group_ops.clear();
  });
}

extern "C" tamm_status tamm_group_end(tamm_ctx* ctx) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!ctx->group_active) throw Error(TAMM_EINVAL, "no contraction group is open");
    std::vector<OzOpRecord> ops;
    ops.swap(ctx->group_ops);
    ctx->group_active = false;
    // every contraction of a group reads inputs that no other one writes, and
    // no two write overlapping outputs: they may then run in any order
    for (size_t i = 0; i < ops.size(); ++i) {
      for (size_t j = 0; j < ops.size(); ++j) {
        if (overlaps(ops[i].c, ops[i].c_bytes, ops[j].left, ops[j].left_bytes) ||
            overlaps(ops[i].c, ops[i].c_bytes, ops[j].right, ops[j].right_bytes))
          throw Error(TAMM_EINVAL, "group: output of contraction %zu overlaps an input of contraction %zu", i, j);
        if (j > i && overlaps(ops[i].c, ops[i].c_bytes, ops[j].c, ops[j].c_bytes))
          throw Error(TAMM_EINVAL, "group: contractions %zu and %zu write overlapping outputs", i, j);
      }
    }
    execute_ozaki(ctx, ops);
  });
}

extern "C" tamm_status tamm_group_cancel(tamm_ctx* ctx) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    if (!ctx->group_active) throw Error(TAMM_EINVAL, "no contraction group is open");
    ctx->group_active = false;
    ctx->group_ops.clear();
  });
}

extern "C" tamm_status tamm_graph_begin(tamm_ctx* ctx) {
  if (!ctx) return TAMM_EINVAL;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (ctx->capturing) throw Error(TAMM_EINVAL, "a graph capture is already open");
    if (ctx->group_active) throw Error(TAMM_EINVAL, "graph capture cannot start inside a contraction group");
    if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy || ctx->stream == cudaStreamPerThread)
      throw Error(TAMM_EINVAL, "graph capture needs the context on a created (non-default) stream");
    if (ctx->profiling) throw Error(TAMM_EINVAL, "switch profiling off before graph capture");
    cuda_check(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    ctx->capturing = true;
    ctx->capture_failed = false;
    ctx->capture_launch0 = ctx->launches;
  });
}

extern "C" tamm_status tamm_graph_end(tamm_ctx* ctx, tamm_graph** out) {
  if (!ctx || !out) return TAMM_EINVAL;
  *out = nullptr;
  return guarded(ctx, [&] {
    require_device(ctx);
    if (!ctx->capturing) throw Error(TAMM_EINVAL, "no graph capture is open");
    if (ctx->group_active) throw Error(TAMM_EINVAL, "close the contraction group before ending the capture");
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->capturing = false;
    for (auto& d : ctx->deferred_graphs) {
      if (d.second) cudaGraphExecDestroy(d.second);
      if (d.first) cudaGraphDestroy(d.first);
    }
    ctx->deferred_graphs.clear();
    const int64_t n = ctx->launches - ctx->capture_launch0;
    if (ctx->capture_failed || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      ctx->capture_failed = false;
      throw Error(e != cudaSuccess ? TAMM_ECUDA : TAMM_EINVAL, "graph capture failed%s%s",
                  e != cudaSuccess ? ": " : " (an operation inside it failed)",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
    }
    std::unique_ptr<tamm_graph> G(new tamm_graph());
    G->ctx = ctx;
    G->graph = g;
    G->launches = n;
    const cudaError_t ei = cudaGraphInstantiate(&G->exec, g, 0);
    if (ei != cudaSuccess) {
      cudaGraphDestroy(g);
      G->graph = nullptr;
      cuda_check(ei, "cudaGraphInstantiate");
    }
    *out = G.release();
  });
}

extern "C" tamm_status tamm_graph_launch(tamm_graph* g) {
  if (!g || !g->ctx) return TAMM_EINVAL;
  tamm_ctx* ctx = g->ctx;
  return guarded(ctx, [&] {
    if (ctx->capturing || ctx->group_active) throw Error(TAMM_EINVAL, "graph launch inside a group or capture");
    cuda_check(cudaGraphLaunch(g->exec, ctx->stream), "cudaGraphLaunch");
    ctx->launches += g->launches;
  });
}

extern "C" tamm_status tamm_graph_info(const tamm_graph* g, int64_t* kernel_launches) {
  if (!g || !kernel_launches) return TAMM_EINVAL;
  *kernel_launches = g->launches;
  return TAMM_OK;
}

extern "C" void tamm_graph_destroy(tamm_graph* g) {
  if (!g) return;
  if (g->ctx && g->ctx->capturing) {  // freed when the open capture ends
    g->ctx->deferred_graphs.emplace_back(g->graph, g->exec);
    delete g;
    return;
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  (void)cudaGetLastError();
  delete g;
}
