// Tensor-core products of strided FP32 matrices (tc_gemm.cu), used by the
// learned correction's network.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mtf {

// a logical matrix of (at least) Rv rows x Kv columns: entry (r, k) at
// X[r sr + k sk]; entries past (Rv, Kv) are zero, except an optional row of
// ones at index ones_r (columns k < Kv) or column of ones at ones_k (rows
// r < Rv) -- the bias of an augmented [W | b] layer
struct TgOperand {
  const float* X = nullptr;
  int64_t sr = 0, sk = 0, Rv = 0, Kv = 0;
  int ones_r = -1, ones_k = -1;
};

// D(r, c) at D[r dr + c dc]; op 0: store, 1: store max(v, 0), 2: store v
// where mask[r mr + c mc] > 0 and 0 elsewhere, 3: add to D; err: the error
// word of the bounded waits of the tensor-core stream
struct TgOut {
  float* D = nullptr;
  int64_t dr = 0, dc = 0;
  int op = 0;
  const float* mask = nullptr;
  int64_t mr = 0, mc = 0;
  unsigned* err = nullptr;
};

struct TcGemm;
TcGemm* tg_create();
void tg_destroy(TcGemm* g);
// D op= A B^T: A is M x K, B is N x K (logical), D is M x N
void tc_gemm(TcGemm& g, const TgOperand& A, const TgOperand& B, int64_t M, int64_t N, int64_t K, const TgOut& out,
             cudaStream_t s);

}  // namespace mtf
