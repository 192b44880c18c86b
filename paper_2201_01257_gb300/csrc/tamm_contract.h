// Contraction layout shared by the FP64 and the split-precision paths.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "tamm_plan.h"

namespace tamm {

constexpr int kMaxLabels = 16;

struct Labels {
  int n = 0;
  char name[kMaxLabels] = {};
  const tamm_space* sp[kMaxLabels] = {};
  int pos[3][kMaxLabels] = {};  // mode position in C / A / B, or -1
  void add(const tamm_tensor* T, const char* l, int which, const char* what);
  int find(char c) const;
};

// Permuted add over a fixed destination/source pair of block tables.
struct AddPlan : Plan {
  AddBlock* d_blocks = nullptr;
  ChunkItem* d_items = nullptr;
  int64_t n_items = 0;
  TileItem* d_tiles = nullptr;  // blocks on the transposition path
  int64_t n_tiles = 0;
  int nm = kMaxKernelModes;
  int n_terms = 1;
  AddPlan(tamm_ctx* c, const tamm_tensor& D, const char* ld, const tamm_tensor& S, int terms, const char* const* ls);
  void run(double* dst, const double* src, double beta, const double* alpha,
           const double* scale_device = nullptr) const;
};

std::vector<AddBlock> build_add_blocks(const tamm_tensor& D, const char* ld, const tamm_tensor& S, int n_terms,
                                       const char* const* ls);
std::vector<ChunkItem> build_chunks(const std::vector<AddBlock>& blocks);

// Roles and nonzero block pairs of C(lc) = beta*C + alpha*A(la)*B(lb).
//   left  = operand holding C's first label; right = the other one
//   need_left  = free_left + summed   (left operand as an M x K matrix per block)
//   need_right = summed + free_right  (right operand as a K x N matrix per block)
//   out_gemm   = free_left + free_right (GEMM output order)
// A *_perm tensor is set when the stored label order differs from the needed one.
struct ContractLayout {
  struct Group {
    int64_t out_block;  // block of the GEMM-order output (out_perm if set, else C)
    int64_t M, N;
    int64_t task_begin, task_end;
  };
  struct Task {
    int64_t left_block, right_block;  // blocks of the GEMM-order operands
    int64_t K;
  };
  Labels L;
  bool swap = false;
  const tamm_tensor* left = nullptr;
  const tamm_tensor* right = nullptr;
  const tamm_tensor* c = nullptr;
  std::string label_left, label_right, label_c;
  std::string free_left, free_right, summed, need_left, need_right, out_gemm;
  std::unique_ptr<tamm_tensor> left_perm, right_perm, out_perm;
  std::vector<Group> groups;
  std::vector<Task> tasks;
  double flops = 0.0;

  ContractLayout(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                 const tamm_tensor* B, const char* lb);
  const tamm_tensor* out_tensor_c() const { return c; }
  const tamm_tensor& left_gemm() const { return left_perm ? *left_perm : *left; }
  const tamm_tensor& right_gemm() const { return right_perm ? *right_perm : *right; }
  const tamm_tensor& out_gemm_tensor() const { return out_perm ? *out_perm : *c; }

 private:
  void enumerate();
};

// slices: integer digit slices (3..8); float_split: BF16x3 floating pieces (slices must be 3).
// Inside a group the contraction is recorded; otherwise it runs at once.
void run_contract_ozaki(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                        const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb, int slices,
                        bool float_split);
// Run recorded split-precision contractions: all slicing, then their GEMMs as few launches as the
// slice counts and the per-launch problem limit allow, then output permutations.
void execute_ozaki(tamm_ctx* ctx, const std::vector<OzOpRecord>& ops);
// Whether the split path may run a contraction through the GEMM that slices A itself (short summed ranges,
// narrow outputs: see ozaki.h).
bool oz_fused_eligible(const ContractLayout& lay);
// Key of a contraction (tensors and labels) in the autotuner's table.
std::string tune_key(const tamm_tensor* C, const char* lc, const tamm_tensor* A, const char* la,
                     const tamm_tensor* B, const char* lb);

}  // namespace tamm
