// Final 2D contraction (Sec. 4: "the remaining two-dimensional network is contracted by
// sweeping an MPS across it"; chi_MPS of Sec. 5) and the coset log-sum / decision.
//
// Site tensor of the final network: F[c][l][r][d][u] = sum_phys R[phys][c] Gamma[phys][..]
// with sqrt(lambda) absorbed on every bond; c is the site's class bit.  Rows y = 0..ny-1 are
// absorbed into a boundary MPS A_x[a][d][b] by zip-up: a carry C[j][a][l][p] runs left to
// right, T[j][u][b][r][q] = sum C A F~ with F~[l,p; r,q] = F[p^q], and (j,u) x (b,r,q) is
// truncated to chi_mps by its leading singular vectors.  The class parity p flows along
// each row into a two-valued output leg of the last MPS tensor.  The last row is contracted
// exactly.
#include <cmath>
#include <mutex>

#include "linalg.cuh"
#include "sweep.cuh"

namespace td {

template <typename R>
__device__ void build_F(const FinalArgs& fa, int b, int x, int y, R* F, int* fd) {
  // fd: dims (L, R, D, U) of the site
  const int s = fa.grid_site[y * fa.nx + x];
  if (s < 0) {
    if (threadIdx.x == 0) { F[0] = R(1); F[1] = R(0); }
    if (threadIdx.x < 4) fd[threadIdx.x] = 1;
    __syncthreads();
    return;
  }
  const FinalSite& fs = fa.sites[s];
  const int dL = fs.dir_dim[0], dR = fs.dir_dim[1], dD = fs.dir_dim[2], dU = fs.dir_dim[3];
  int stride[kMaxBonds];
  {
    int st = 1;
    for (int k = fs.nb - 1; k >= 0; --k) {
      stride[k] = st;
      int dk = 1;
      for (int dir = 0; dir < 4; ++dir)
        if (fs.dir_pos[dir] == k) dk = fs.dir_dim[dir];
      st *= dk;
    }
  }
  int rest = 1;
  for (int dir = 0; dir < 4; ++dir) rest *= fs.dir_dim[dir];
  const int64_t shot = (int64_t)b * fa.shot_elems;
  const double* lam = fa.lam + (int64_t)b * fa.nbonds * fa.chi;
  const int n = dL * dR * dD * dU;
  for (int w = threadIdx.x; w < 2 * n; w += blockDim.x) {
    const int c = w / n;
    int e = w % n;
    const int iu = e % dU; e /= dU;
    const int id = e % dD; e /= dD;
    const int ir = e % dR; e /= dR;
    const int il = e;
    const int idx[4] = {il, ir, id, iu};
    int64_t off = 0;
    R wgt = R(1);
    for (int dir = 0; dir < 4; ++dir)
      if (fs.dir_pos[dir] >= 0) {
        off += (int64_t)idx[dir] * stride[fs.dir_pos[dir]];
        wgt *= R(sqrt(lam[fs.dir_bond[dir] * fa.chi + idx[dir]]));
      }
    R acc = R(0);
    for (int ph = 0; ph < fs.P; ++ph) {
      const double rr = fs.R[ph * 2 + c];
      if (rr == 0.0) continue;
      R g = reinterpret_cast<const R*>(fa.gamma)[shot + fs.off + (int64_t)ph * rest + off];
      acc += R(rr) * g;
    }
    F[w] = acc * wgt;
  }
  if (threadIdx.x == 0) { fd[0] = dL; fd[1] = dR; fd[2] = dD; fd[3] = dU; }
  __syncthreads();
}

template <typename R>
__global__ void k_final(FinalArgs fa) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  R* scr = reinterpret_cast<R*>(fa.scratch) + (int64_t)b * fa.scratch_elems;
  R* mps[2] = {scr + fa.off_mps0, scr + fa.off_mps1};
  R* Cb[2] = {scr + fa.off_C0, scr + fa.off_C1};
  R* F = scr + fa.off_F;
  R* T1 = scr + fa.off_T1;
  R* Tm = scr + fa.off_T;
  R* G = scr + fa.off_G;
  R* V = scr + fa.off_V;
  R* sv = scr + fa.off_s;
  __shared__ int mdim[2][32][3];   // per column: (left, down, right) of the MPS tensors
  __shared__ int fd[4];
  __shared__ int meta[8];
  __shared__ R rot[2 * 160];
  __shared__ int order_s[1];
  __shared__ double logsum_s;
  const int nx = fa.nx, ny = fa.ny;
  if (tid == 0) logsum_s = 0.0;
  for (int x = tid; x < nx; x += nt) {
    mdim[0][x][0] = 1; mdim[0][x][1] = 1; mdim[0][x][2] = (x == nx - 1) ? 2 : 1;
    R* A = mps[0] + (int64_t)x * fa.mps_stride;
    A[0] = R(1);
    if (x == nx - 1) A[1] = R(0);
  }
  __syncthreads();
  int cur = 0;
  for (int y = 0; y < ny; ++y) {
    int cc = 0;
    // carry C[j][a][l][p]: j = 1, a = 1, l = 1, p = 0
    if (tid == 0) { Cb[0][0] = R(1); Cb[0][1] = R(0); }
    int cJ = 1, cA = 1, cL = 1;
    __syncthreads();
    for (int x = 0; x < nx; ++x) {
      build_F<R>(fa, b, x, y, F, fd);
      const int L = fd[0], Rr = fd[1], Dd = fd[2], U = fd[3];
      const R* A = mps[cur] + (int64_t)x * fa.mps_stride;
      const int aL = mdim[cur][x][0], aD = mdim[cur][x][1], aR = mdim[cur][x][2];
      const R* C = Cb[cc];
      // T1[j][l][p][d][bb] = sum_a C[j][a][l][p] A[a][d][bb]   (a: cA == aL, d: Dd == aD, l: cL == L)
      const int n1 = cJ * L * 2 * aD * aR;
      for (int w = tid; w < n1; w += nt) {
        int e = w;
        const int bb = e % aR; e /= aR;
        const int d = e % aD; e /= aD;
        const int p = e % 2; e /= 2;
        const int l = e % L; e /= L;
        const int j = e;
        R acc = R(0);
        for (int a = 0; a < aL; ++a) acc += C[((j * cA + a) * cL + l) * 2 + p] * A[(a * aD + d) * aR + bb];
        T1[w] = acc;
      }
      __syncthreads();
      // Tm[j][u][bb][r][q] = sum_{l,p,d} T1[j][l][p][d][bb] F[p^q][l][r][d][u]
      const int nF = L * Rr * Dd * U;
      const int n2 = cJ * U * aR * Rr * 2;
      for (int w = tid; w < n2; w += nt) {
        int e = w;
        const int q = e % 2; e /= 2;
        const int r = e % Rr; e /= Rr;
        const int bb = e % aR; e /= aR;
        const int u = e % U; e /= U;
        const int j = e;
        R acc = R(0);
        for (int l = 0; l < L; ++l)
          for (int p = 0; p < 2; ++p)
            for (int d = 0; d < aD; ++d)
              acc += T1[(((j * L + l) * 2 + p) * aD + d) * aR + bb] * F[(p ^ q) * nF + ((l * Rr + r) * Dd + d) * U + u];
        Tm[w] = acc;
      }
      __syncthreads();
      R* An = mps[cur ^ 1] + (int64_t)x * fa.mps_stride;
      const int m = cJ * U, n = aR * Rr * 2;
      if (x < nx - 1 && y < ny - 1) {
        // SVD of M = Tm [(j,u) x (b,r,q)] by one-sided Jacobi on the rows of M: the columns
        // of MT = M^T are orthogonalised, MT W = (S V^T)^T, W = left singular vectors.
        R* MT = G;
        for (int w = tid; w < m * n; w += nt) {
          const int ju = w / n, c = w % n;
          MT[c * m + ju] = Tm[w];
        }
        __syncthreads();
        block_svd_onesided<R>(MT, m, n, m, V, m, rot, meta + 7);
        int* ord = reinterpret_cast<int*>(Tm + m * n);   // scratch after Tm (sized on host)
        for (int j = tid; j < m; j += nt) {
          R s2 = R(0);
          for (int c = 0; c < n; ++c) s2 += MT[c * m + j] * MT[c * m + j];
          sv[m + j] = sqrt(s2);
        }
        __syncthreads();
        if (tid == 0) {
          for (int i = 0; i < m; ++i) ord[i] = i;
          for (int i = 1; i < m; ++i) {
            int xk = ord[i], k = i - 1;
            while (k >= 0 && sv[m + ord[k]] < sv[m + xk]) { ord[k + 1] = ord[k]; --k; }
            ord[k + 1] = xk;
          }
          for (int i = 0; i < m; ++i) sv[i] = sv[m + ord[i]];
          int k = 0;
          const int nsv = m < n ? m : n;
          if (sv[0] > R(0)) k = keep_count<R>(sv, nsv, fa.chi_mps, fa.svd_cutoff, fa.multiplet_rtol);
          meta[0] = k;
        }
        __syncthreads();
        const int k = meta[0];
        if (k == 0) {
          if (tid == 0) logsum_s = -INFINITY;
          // keep a single zero column so shapes stay valid
          for (int w = tid; w < m; w += nt) An[w] = R(0);
          R* Cn = Cb[cc ^ 1];
          for (int w = tid; w < n; w += nt) Cn[w] = R(0);
          __syncthreads();
          if (tid == 0) { mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = 1; }
          cJ = 1;
        } else {
          const R s0 = sv[0];
          for (int w = tid; w < m * k; w += nt) {
            const int ju = w / k, kk = w % k;
            An[w] = V[ju * m + ord[kk]];            // An[j][u][kk]
          }
          R* Cn = Cb[cc ^ 1];
          for (int w = tid; w < k * n; w += nt) {
            const int kk = w / n, c = w % n;
            Cn[w] = MT[c * m + ord[kk]] / s0;       // Cn[kk][bb][r][q] = (S V^T)[kk][c] / s0
          }
          if (tid == 0) {
            logsum_s += log((double)s0);
            mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = k;
          }
          cJ = k;
        }
        cA = aR; cL = Rr;
        cc ^= 1;
        __syncthreads();
      } else if (x < nx - 1) {
        // last row: U == 1, no truncation; the carry takes the whole contraction
        R* Cn = Cb[cc ^ 1];
        for (int w = tid; w < m * n; w += nt) Cn[w] = Tm[w];
        for (int w = tid; w < m * m; w += nt) An[w] = (w / m == w % m) ? R(1) : R(0);
        if (tid == 0) { mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = m; }
        cJ = m; cA = aR; cL = Rr;
        cc ^= 1;
        __syncthreads();
      } else {
        // last column: merge the old class leg bb and the row parity q into c' = bb ^ q
        if (tid == 0) {
          R mx = R(0);
          for (int ju = 0; ju < m; ++ju)
            for (int c2 = 0; c2 < 2; ++c2) {
              R acc = R(0);
              for (int bb = 0; bb < aR; ++bb)
                for (int q = 0; q < 2; ++q)
                  if ((bb ^ q) == c2) acc += Tm[((ju * aR + bb) * Rr + 0) * 2 + q];
              An[ju * 2 + c2] = acc;
              mx = fmax(mx, fabs(acc));
            }
          if (mx > R(0)) {
            for (int w = 0; w < m * 2; ++w) An[w] /= mx;
            logsum_s += log((double)mx);
          } else {
            logsum_s = -INFINITY;
          }
          mdim[cur ^ 1][x][0] = cJ; mdim[cur ^ 1][x][1] = U; mdim[cur ^ 1][x][2] = 2;
        }
        __syncthreads();
      }
    }
    cur ^= 1;
    __syncthreads();
  }
  if (tid == 0) {
    // contract the last MPS (vertical legs are trivial): v <- v A_x
    R v[64], vn[64];
    v[0] = R(1);
    int dv = 1;
    for (int x = 0; x < nx; ++x) {
      const R* A = mps[cur] + (int64_t)x * fa.mps_stride;
      const int aL = mdim[cur][x][0], aR = mdim[cur][x][2];
      for (int bb = 0; bb < aR && bb < 64; ++bb) {
        R acc = R(0);
        for (int a = 0; a < aL && a < dv; ++a) acc += v[a] * A[a * aR + bb];
        vn[bb] = acc;
      }
      dv = aR < 64 ? aR : 64;
      for (int bb = 0; bb < dv; ++bb) v[bb] = vn[bb];
    }
    fa.Z[(int64_t)b * 2 + 0] = double(v[0]);
    fa.Z[(int64_t)b * 2 + 1] = double(v[1]);
    fa.logacc[(int64_t)b * fa.nslots + fa.slot] = logsum_s;
  }
}

__global__ void k_finalize(FinalizeArgs f) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= f.B) return;
  double ls = 0.0;
  for (int k = 0; k < f.nslots; ++k) ls += f.logacc[(int64_t)b * f.nslots + k];
  const double z0 = f.Z[2 * b], z1 = f.Z[2 * b + 1];
  double zz[2] = {f.mix[0] * z0 + f.mix[1] * z1, f.mix[2] * z0 + f.mix[3] * z1};
  int off = 0;
  if (f.offset_all) {
    const uint8_t* m = f.det + (int64_t)(f.wave_first + b) * f.n_det;
    for (int i = 0; i < f.n_det; ++i) off ^= m[i] & 1;
  }
  double lp[2];
  for (int c = 0; c < 2; ++c) {
    const double z = zz[c ^ off];
    lp[c] = (z > 0.0 && ls > -INFINITY) ? log(z) + ls : -INFINITY;
  }
  const int64_t gb = f.wave_first + b;
  if (f.logp) {
    f.logp[2 * gb] = lp[0];
    f.logp[2 * gb + 1] = lp[1];
  }
  const int dec = (lp[1] > lp[0]) ? 1 : 0;
  if (f.decision) f.decision[gb] = dec;
  if (f.margin) f.margin[gb] = lp[dec] - lp[dec ^ 1];
}

template <typename T, typename R>
cudaError_t launch_final(const FinalArgs& f, cudaStream_t st) {
  k_final<R><<<f.B, 256, 0, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& f, cudaStream_t st) {
  k_finalize<<<(f.B + 127) / 128, 128, 0, st>>>(f);
  return cudaGetLastError();
}

// ---- final contraction with scratch in a static device array ----------------------------
// For callers that cannot call cudaMalloc: the scratch of k_final comes from this
// file-scope array instead of the network workspace.  Every GPU that loads the library holds
// it until the process exits.  Host code must not use the symbol as an address; the device
// address is looked up once per device (cudaGetSymbolAddress) with that device current.
static __device__ __align__(256) unsigned char g_final_scratch[kStaticFinalScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices] = {};
}  // namespace

cudaError_t static_final_scratch(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxStaticDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_final_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *ptr = g_static_ptr[dev];
  return cudaSuccess;
}

template cudaError_t launch_final<double, double>(const FinalArgs&, cudaStream_t);
template cudaError_t launch_final<float, float>(const FinalArgs&, cudaStream_t);

}  // namespace td
