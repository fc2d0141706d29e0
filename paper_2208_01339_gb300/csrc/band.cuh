// Exact A_f^{-1} for fracture blocks of any geometry (internal).
//
// The paper factors A once with an exact sparse Cholesky and applies
// A^{-1} by triangular solves (Section 4.2, Algorithm 3).  Here each
// fracture block A_f is reordered on the host (reverse Cuthill-McKee, or
// the caller's numbering when that gives the narrower band), factored on
// the GPU as a band matrix of half-bandwidth w_f, and used twice:
//   * M_f = (A_f^{-1}) restricted to trace rows and columns, one dense block
//     per fracture, from multi-right-hand-side band solves with the unit
//     vectors of the trace nodes (the Schur operator and Algorithm 4 then
//     run on M exactly as for the closed-form rectangles);
//   * full solves y = A^{-1} v (right-hand side, recovery of h and p).
//
// Band storage: row i of the factor of fracture f holds L(i, i-w..i) at
// L[boff[f] + i (w+1) + w - i + j], the diagonal last; entries left of
// column 0 are zero.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace pp {

constexpr int kBandMaxW = 768;   // largest half-bandwidth accepted after reordering
constexpr int kBandCols = 32;    // trace columns per work item of the M build
constexpr int kBandWarps = 8;    // warps of the M-build block (split the band)
constexpr int kPanel = 8;        // columns per panel of the factorisation
constexpr int kPanelStride = 9;  // doubles per row of the panel buffer (padded against bank conflicts)

// Doubles of the factorisation window of a block with W = w + 1: the live
// rows of the band (W + kPanel - 1 of them) folded into a packed triangle,
// then the panel buffer.
__host__ __device__ inline long long factor_window_doubles(int W) {
  const long long WP = (long long)W + kPanel - 1;
  return WP * (WP + 1) / 2 + WP * kPanelStride;
}

struct BandHost {
  int n_f = 0, max_w = 0, max_n = 0, n_items = 0, rcm_used = 0;
  long long elems = 0, gwin_elems = 0;
  size_t factor_smem = 0;           // dynamic shared memory of the factor launch
  std::vector<int> w;               // half-bandwidth per fracture
  std::vector<int> rcm;             // 1 where reverse Cuthill-McKee beat the given numbering
  std::vector<long long> boff;      // band storage offsets (n_f + 1)
  std::vector<long long> gwoff;     // factor window in global memory (-1: shared memory)
  std::vector<int> pos;             // n_h: position of each node in its fracture's order
  std::vector<int> perm;            // n_h: local node at offset[f] + position
  std::vector<int> trace_at;        // n_h: local trace index at offset[f] + position, or -1
  std::vector<int> order;           // fractures by decreasing factorisation work
  std::vector<int> tcol, tpos;      // n_T: trace columns per fracture sorted by position
  std::vector<int> tposa;           // n_T: position of each trace node (by local trace index)
  std::vector<int4> items;          // (fracture, first slot, count, first position)
};

struct BandDev {
  int n_f = 0, max_w = 0, max_n = 0, n_items = 0, grid_trace = 0;
  size_t factor_smem = 0;
  const long long* off = nullptr;   // fracture row offsets (n_f + 1)
  const int* w = nullptr;
  const long long* boff = nullptr;
  const long long* gwoff = nullptr;
  const int *pos = nullptr, *perm = nullptr, *trace_at = nullptr, *order = nullptr;
  const int *tcol = nullptr, *tpos = nullptr, *tposa = nullptr;
  const int4* items = nullptr;
  double* L = nullptr;
  double* dinv = nullptr;           // n_h: 1 / L(i, i) by fracture position
  double* gwin = nullptr;
  double* Z = nullptr;              // grid_trace x max_n x kBandCols forward results
  int* flags = nullptr;             // [0] first non-positive pivot + 1, [1] work-queue counter
};

// Host plan.  A: host CSR (n_h rows, global numbering) of the block-diagonal
// fracture matrix; toff/tnode: trace nodes per fracture (tnode ascending).
// Returns 0 or a PP_* status with err set.
int band_plan(int n_f, int n_h, const long long* offset, const std::vector<int>& rp, const std::vector<int>& col,
              const std::vector<double>& val, const std::vector<long long>& toff, const std::vector<int>& tnode,
              BandHost& H, std::string& err);

// Bytes of opt-in shared memory a block may use on this device.
size_t band_smem_optin();

// Scatter A into the (zeroed) band storage.
cudaError_t band_fill(const BandDev& D, int n_h, const int* rp, const int* col, const double* val, cudaStream_t s);
// L_f L_f^T = A_f for every fracture; flags[0] = first failing fracture + 1.
cudaError_t band_factor(const BandDev& D, cudaStream_t s);
// M_f[a][b] = (A_f^{-1})[trace a][trace b] for every fracture.
cudaError_t band_trace_blocks(const BandDev& D, const long long* toff, const long long* moff, double* M,
                              cudaStream_t s);
// y = A^{-1} v (n_h vectors, global numbering); z: n_h scratch.  y may alias v.
cudaError_t band_solve(const BandDev& D, int n_h, const double* v, double* y, double* z, cudaStream_t s);

}  // namespace pp
