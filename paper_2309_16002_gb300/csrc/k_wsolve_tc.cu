// Interpolation matrix of Alg. 3 on Blackwell tensor cores (sm_103a): the
// block-inverse factors and the launch of the solve.
//
// W L1 = L with L1 = L(S, :) lower triangular (Sec. 5.1) is solved by blocks
// of 64 columns.  With J = [j0, j0 + 64), J+ = [j0 + 64, k) and T_J = L1(J, J):
//   W(:, J) = (L(:, J) - W(:, J+) L1(J+, J)) T_J^{-1}
//           = L(:, J) G(J, J) + W(:, J+) G(J+, J),
//   G(J, J) = T_J^{-1},  G(J+, J) = -L1(J+, J) T_J^{-1}.
// k_wsolve_g forms G once (FP32; one 64-wide row solve with T_J per row of G),
// stored transposed and split into TF32 hi/lo, so that every term of W is a
// tensor-core product and no substitution runs on the n rows of W; the
// right-looking solve that takes those products is k_wsolve_rl (k_wsolve_rl.cu).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "rbrp_internal.cuh"
#include "tc_common.cuh"

namespace rbrp {
namespace tc {

constexpr int WM = 128;  // rows per tile of the solve
constexpr int WN = 64;   // column block

// Rows r0 .. r0 + 127 of G(:, J), one CTA per (row block, J).  Row r solves
// y T_J = rhs with rhs = e_(r - j0) for r in J (then G(r, J) = y) and
// rhs = L1(r, J) for r past J (then G(r, J) = -y), by back substitution over
// the columns of y from the last, each finished y_c updating the earlier
// right-hand sides.  FP32; the result is stored transposed and split for the
// MMA B operand: Gh/Gl[(j0 + c) * ldt + r].
__global__ void __launch_bounds__(128) k_wsolve_g(const double* __restrict__ L1, long long ld1, int k,
                                                  float* __restrict__ Gh, float* __restrict__ Gl, long long ldt) {
  pdl_wait();
  const int J = blockIdx.y, j0 = J * WN;
  const int r0 = blockIdx.x * 128;
  if (r0 + 128 <= j0 || r0 >= k) return;
  const int nb = min(WN, k - j0);
  __shared__ __align__(16) float Ts[WN][WN];  // Ts[c][a] = L1(j0 + c, j0 + a) for a < c < nb, else 0
  __shared__ float rinv[WN];
  for (int e = threadIdx.x; e < WN * WN; e += 128) {
    const int c = e / WN, a = e % WN;
    Ts[c][a] = (a < c && c < nb) ? (float)L1[(long long)(j0 + c) * ld1 + j0 + a] : 0.f;
  }
  if (threadIdx.x < WN) {
    const int c = threadIdx.x;
    rinv[c] = c < nb ? (float)(1.0 / L1[(long long)(j0 + c) * ld1 + j0 + c]) : 0.f;
  }
  __syncthreads();
  const int r = r0 + threadIdx.x;
  if (r < j0 || r >= k) return;
  const bool in_J = r < j0 + nb;
  float y[WN];
#pragma unroll
  for (int c = 0; c < WN; ++c)
    y[c] = in_J ? (c == r - j0 ? 1.f : 0.f) : (c < nb ? (float)L1[(long long)r * ld1 + j0 + c] : 0.f);
#pragma unroll
  for (int c = WN - 1; c >= 0; --c) {
    const float yc = y[c] * rinv[c];
    y[c] = yc;
#pragma unroll
    for (int a = 0; a + 4 <= c; a += 4) {
      const float4 t = *(const float4*)&Ts[c][a];
      y[a] -= yc * t.x;
      y[a + 1] -= yc * t.y;
      y[a + 2] -= yc * t.z;
      y[a + 3] -= yc * t.w;
    }
#pragma unroll
    for (int a = c & ~3; a < c; ++a) y[a] -= yc * Ts[c][a];
  }
  const float sg = in_J ? 1.f : -1.f;
#pragma unroll
  for (int c = 0; c < WN; ++c) {
    if (c < nb) {
      const float v = sg * y[c];
      const float h = tf32_rn(v);
      Gh[(long long)(j0 + c) * ldt + r] = h;
      Gl[(long long)(j0 + c) * ldt + r] = tf32_rn(v - h);
    }
  }
}

template <bool L64>
cudaError_t wsolve_rl(const void* L, long long ldl, double* W64, long long ldw64, float* Wb, long long ldwb,
                      const float* Gh, const float* Gl, long long ldt, long long r0, long long r1, long long k,
                      State* st, cudaStream_t s);

}  // namespace tc

cudaError_t launch_wsolve_tc(const void* L, int l_is_fp64, long long ldl, float* Wb, long long ldwb, double* W64,
                             long long ldw64, const double* L1, long long ld1, float* Gh, float* Gl, long long ldt,
                             long long n, long long r0, long long r1, bool form_g, long long k, State* st,
                             cudaStream_t s) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  if (r0 < 0 || r1 > n || r0 % tc::WM != 0) return cudaErrorInvalidValue;
  if (form_g) {
    const int nblk = (int)((k + tc::WN - 1) / tc::WN);
    cudaError_t e = launch_pdl(tc::k_wsolve_g, dim3((unsigned)((k + 127) / 128), (unsigned)nblk), dim3(128), 0, s, L1,
                               ld1, (int)k, Gh, Gl, ldt);
    if (e != cudaSuccess) return e;
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
  }
  if (r1 <= r0) return cudaSuccess;
  if (l_is_fp64) return tc::wsolve_rl<true>(L, ldl, W64, ldw64, Wb, ldwb, Gh, Gl, ldt, r0, r1, k, st, s);
  return tc::wsolve_rl<false>(L, ldl, W64, ldw64, Wb, ldwb, Gh, Gl, ldt, r0, r1, k, st, s);
}

int wsolve_tc_rows_per_tile() { return tc::WM; }

}  // namespace rbrp
