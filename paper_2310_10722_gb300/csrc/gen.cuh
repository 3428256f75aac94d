// Kernels of generator networks (gen.cu): syndromes to sweep rows, rows to classes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace td {

struct GenRowsArgs {
  const uint8_t* syn;                 // [B][n_checks] syndromes
  int64_t B;
  int32_t n_checks, words;            // words = 64-bit words per packed syndrome
  const unsigned long long* trans;    // [n_checks + 1][words] elimination transform rows
  int32_t rank;
  const int32_t* col;                 // [rank] row column of pivot i
  const uint8_t* xbar;                // [n_cols] xbar in column order
  int32_t n_cols;                     // row length (qubits)
  uint8_t* rows;                      // [2B][n_cols] out: r, r + xbar
  int32_t* cls;                       // [B] out: class of r, -1 if m is not a syndrome
};

struct GenCombineArgs {
  const double* row_logp;             // [2B][2] contractions of the rows (class-0 entry used)
  const int32_t* cls;                 // [B]
  int64_t B;
  double log_offset;                  // -(n_gen - rank of the generators) ln 2
  double* logp;                       // [B][2] or null
  int32_t* decision;                  // [B] or null
  double* margin;                     // [B] or null
};

cudaError_t launch_gen_rows(const GenRowsArgs& g, cudaStream_t st);
cudaError_t launch_gen_combine(const GenCombineArgs& g, cudaStream_t st);

}  // namespace td
