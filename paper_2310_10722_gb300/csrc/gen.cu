// Generator networks (Sec. 3.2): from syndromes to the rows of the sweep, and from the
// rows' contractions back to the two classes.
//
// The representative r of a syndrome m (the error supported on the greedy column basis of H
// with H r = m) is linear in m: row i < rank of the build-time elimination transform gives
// r's bit at column col[i] as a GF(2) dot product with m, rows rank .. n_checks-1 vanish
// exactly when m is a syndrome, and the last row gives the class r . zbar.  A shot becomes
// two rows of the sweep, r and r + xbar (the cosets of both classes).
#include <cmath>

#include "gen.cuh"

namespace td {

namespace {
constexpr int kGenWarps = 8;   // shots per block, one warp each
}

// One warp per shot.  Dynamic shared memory: the packed syndrome of each warp (words words).
__global__ void __launch_bounds__(kGenWarps * 32) k_gen_rows(GenRowsArgs g) {
  extern __shared__ unsigned long long sm_words[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kGenWarps + warp;
  if (b >= g.B) return;
  unsigned long long* mw = sm_words + (size_t)warp * g.words;
  const uint8_t* m = g.syn + b * g.n_checks;
  uint8_t* r0 = g.rows + 2 * b * g.n_cols;
  uint8_t* r1 = r0 + g.n_cols;
  // pack the syndrome, 64 checks per word (bits outside {0,1} count by their low bit)
  for (int w = lane; w < g.words; w += 32) {
    unsigned long long v = 0ull;
    const int c0 = w * 64;
    for (int k = 0; k < 64 && c0 + k < g.n_checks; ++k) v |= (unsigned long long)(m[c0 + k] & 1) << k;
    mw[w] = v;
  }
  for (int j = lane; j < g.n_cols; j += 32) r0[j] = 0;
  __syncwarp();
  auto dot = [&](int i) {
    const unsigned long long* row = g.trans + (int64_t)i * g.words;
    int par = 0;
    for (int w = 0; w < g.words; ++w) par ^= __popcll(row[w] & mw[w]);
    return par & 1;
  };
  for (int i = lane; i < g.rank; i += 32)
    if (dot(i)) r0[g.col[i]] = 1;
  int bad = 0;
  for (int i = g.rank + lane; i < g.n_checks; i += 32) bad |= dot(i);
  bad = __any_sync(0xffffffffu, bad);
  const int cls = dot(g.n_checks);
  __syncwarp();
  for (int j = lane; j < g.n_cols; j += 32) r1[j] = r0[j] ^ g.xbar[j];
  if (lane == 0) g.cls[b] = bad ? -1 : cls;
}

// One thread per shot: log p_{m, cls ^ c} = the contraction of row 2b + c (its class-0
// entry; a generator network's rows carry no class leg) plus the dependency offset.
__global__ void k_gen_combine(GenCombineArgs g) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.B) return;
  const int cls = g.cls[b];
  double lp[2];
  if (cls < 0) {
    lp[0] = lp[1] = -INFINITY;
  } else {
    for (int c = 0; c < 2; ++c) {
      const double v = g.row_logp[(2 * b + c) * 2];
      lp[cls ^ c] = (v > -INFINITY) ? v + g.log_offset : v;
    }
  }
  if (g.logp) {
    g.logp[2 * b] = lp[0];
    g.logp[2 * b + 1] = lp[1];
  }
  const int dec = (lp[1] > lp[0]) ? 1 : 0;
  if (g.decision) g.decision[b] = dec;
  if (g.margin) g.margin[b] = lp[dec] - lp[dec ^ 1];
}

cudaError_t launch_gen_rows(const GenRowsArgs& g, cudaStream_t st) {
  if (g.B == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((g.B + kGenWarps - 1) / kGenWarps);
  const size_t smem = (size_t)kGenWarps * g.words * sizeof(unsigned long long);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gen_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gen_rows<<<blocks, kGenWarps * 32, smem, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_gen_combine(const GenCombineArgs& g, cudaStream_t st) {
  if (g.B == 0) return cudaSuccess;
  k_gen_combine<<<(unsigned)((g.B + 127) / 128), 128, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace td
