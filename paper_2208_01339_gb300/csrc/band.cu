// Banded Cholesky factors of general fracture blocks and the solves built on
// them (declarations and storage in band.cuh).
//
// Factorisation: one block per fracture, in panels of kPanel columns.  The
// panel's columns are scaled by their pivots and update the panel's later
// columns one by one; then the triangle below the panel takes one rank-kPanel
// update, each entry read and written once for kPanel FMAs.  The live part of
// the band -- rows jp..jp+w+kPanel-1 for the panel starting at column jp,
// columns jp..i of row i -- is kept in a window indexed by (row mod WP,
// column mod WP), WP = w + kPanel.  Of the two mirrored slots (a, b) and
// (b, a) only one is live at any time, so the window folds into a packed
// triangle of WP (WP + 1) / 2 doubles.  For w <= 225 it fits in shared
// memory; wider bands keep the same window in global memory.  Every band
// entry is read from HBM once and the factor written once.
//
// Trace blocks: work item = one fracture and up to 32 of its trace columns
// (sorted by position, so the forward solve starts at the first one: the
// unit vectors are zero above it).  Lanes are columns, warps split the band.
// Forward L y = e in dot form over row i of L; backward L^T x = y in axpy form
// over the same row (x_i is final once rows i+1..i+w have been applied), so
// both sweeps read L by rows.  The backward sweep also stops at the first
// column: M_f is symmetric, and an entry above it is the mirror of one the
// earlier column computes.  Rows of x that are trace nodes are written into
// M_f.  Items are handed out largest first from a device counter.
//
// Full solves: one warp per fracture, the same two sweeps on one vector.
//
// The sweeps are latency chains (row i needs row i-1), so the rows of the
// factor they read -- with the pivot reciprocals and the vector entries of
// the same step -- are copied into shared memory a few rows ahead with
// cp.async.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>

#include "../../include/polyprec.h"
#include "band.cuh"
#include "common.cuh"
#include "driver.cuh"

namespace pp {
namespace {

__host__ __device__ __forceinline__ int tri(int a) { return (a * (a + 1)) >> 1; }

// packed window slot of the live entry (i, j), i >= j
__device__ __forceinline__ int wslot(int i, int j, int W) {
  const int a = i % W, b = j % W;
  return a >= b ? tri(a) + b : tri(b) + a;
}

__device__ __forceinline__ int fracture_of(const long long* off, int nf, long long e) {
  int lo = 0, hi = nf;  // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void band_fill_kernel(BandDev D, int n_h, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_h;
       r += (long long)gridDim.x * blockDim.x) {
    const int f = fracture_of(D.off, D.n_f, r);
    const int w = D.w[f], W = w + 1;
    const int pi = D.pos[r];
    double* row = D.L + D.boff[f] + (long long)pi * W + w - pi;  // row[pj] = (pi, pj)
    for (int p = rp[r]; p < rp[r + 1]; ++p) {
      const int pj = D.pos[col[p]];
      if (pj <= pi) row[pj] = val[p];
    }
  }
}

constexpr int kFactorThreads = 512;
constexpr int kRowsAhead = 4;  // band rows in flight (cp.async ring) in the solve sweeps

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The factorisation of fracture f with its window at `win` (shared memory
// for SH, else global): instantiated twice so that the shared-memory case
// addresses the window with 32-bit shared loads and stores.
template <bool SH>
__device__ __forceinline__ void factor_block(const BandDev& D, int f, double* win) {
  const long long o = D.off[f];
  const int n = (int)(D.off[f + 1] - o), w = D.w[f], W = w + 1;
  const int WP = W + kPanel - 1;  // live rows: a panel's columns reach w rows below its last one
  double* L = D.L + D.boff[f];
  double* dinv = D.dinv + o;
  double* P = win + tri(WP);  // P[(i - jp) kPanelStride + c] = L(i, jp + c) for the current panel
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nt = kFactorThreads, nw = kFactorThreads / 32;
  // rows 0..WP-1 are all live at the first panel
  const int r0 = min(WP - 1, n - 1);
  for (int i = 0; i <= r0; ++i)
    for (int k = max(0, i - w) + tid; k <= i; k += nt) win[wslot(i, k, WP)] = L[(long long)i * W + w - i + k];
  __syncthreads();
  bool bad = false;
  for (int jp = 0; jp < n; jp += kPanel) {
    const int nbb = min(kPanel, n - jp);
    for (int e = tid; e < WP * kPanelStride; e += nt) P[e] = 0.0;
    __syncthreads();
    // the panel, column by column: scale, then update the panel's later columns
    for (int cc = 0; cc < nbb; ++cc) {
      const int c = jp + cc;
      const double acc = win[wslot(c, c, WP)];
      const bool ok = acc > 0.0;  // false for NaN too
      bad |= !ok;
      const double d = ok ? sqrt(acc) : 1.0;
      const double rd = 1.0 / d;
      const int m = min(w, n - 1 - c);
      for (int r = 1 + tid; r <= m; r += nt) {
        const double l = win[wslot(c + r, c, WP)] * rd;
        P[(c + r - jp) * kPanelStride + cc] = l;
        L[(long long)(c + r) * W + w - r] = l;
      }
      if (tid == 0) {
        L[(long long)c * W + w] = d;
        dinv[c] = rd;
      }
      __syncthreads();
      const int rem = min(nbb - 1 - cc, m);  // later panel columns c + s, s <= rem, inside the band
      if (rem > 0) {
        for (int e = tid; e < rem * m; e += nt) {
          const int s = 1 + e % rem, r = 1 + e / rem;
          if (s > r) continue;
          const int idx = wslot(c + r, c + s, WP);
          win[idx] = fma(-P[(c + r - jp) * kPanelStride + cc], P[(c + s - jp) * kPanelStride + cc], win[idx]);
        }
      }
      __syncthreads();
    }
    // rank-nbb update of the trailing triangle: rows and columns K0..R1.
    // Work item = 32 columns (one per lane) x 8 rows; each lane keeps its
    // column's panel values in registers, the row's are a broadcast load.
    const int K0 = jp + nbb, R1 = min(jp + nbb - 1 + w, n - 1);
    const int mt = R1 - K0 + 1;
    if (mt > 0) {
      const int strips = (mt + 31) >> 5;
      int s = 0, base = 0;  // items of the strips before s
      for (int it = warp;; it += nw) {
        while (s < strips && it >= base + ((mt - 32 * s + 7) >> 3)) {
          base += (mt - 32 * s + 7) >> 3;
          ++s;
        }
        if (s >= strips) break;
        const int k = K0 + 32 * s + lane;
        const int i0 = K0 + 32 * s + 8 * (it - base), i1 = min(i0 + 8, R1 + 1);
        if (k <= R1) {
          double pk[kPanel];
#pragma unroll
          for (int q = 0; q < kPanel; ++q) pk[q] = P[(k - jp) * kPanelStride + q];
          for (int i = max(i0, k); i < i1; ++i) {
            const double* pi = P + (i - jp) * kPanelStride;
            const int idx = wslot(i, k, WP);
            double v = win[idx];
#pragma unroll
            for (int q = 0; q < kPanel; ++q) v = fma(-pi[q], pk[q], v);
            win[idx] = v;
          }
        }
      }
    }
    // rows jp+WP.. enter in the slots the panel's columns have left
    for (int q = tid; q < nbb * W; q += nt) {
      const int inew = jp + WP + q / W, cq = q % W;
      if (inew < n) win[wslot(inew, inew - w + cq, WP)] = L[(long long)inew * W + cq];
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicCAS(D.flags, 0, f + 1);
}

__global__ void __launch_bounds__(kFactorThreads, 1) band_factor_kernel(BandDev D) {
  extern __shared__ double band_sm[];
  const int f = D.order[blockIdx.x];
  if (D.gwoff[f] < 0)
    factor_block<true>(D, f, band_sm);
  else
    factor_block<false>(D, f, D.gwin + D.gwoff[f]);
}

// Shared-memory layout of the M-build block: partial sums, the broadcast
// x row, the W x NC ring of the sweep, and kRowsAhead row buffers of
// stride max_w + 2 + NC: L(row, row-w..row), 1/L(row,row) and, in the
// backward sweep, the NC forward values of row - W.
__host__ __device__ inline size_t trace_smem_doubles(int max_w) {
  const size_t W = (size_t)max_w + 1;
  return (size_t)kBandWarps * kBandCols + kBandCols + W * kBandCols + kRowsAhead * (W + 1 + kBandCols);
}

__global__ void __launch_bounds__(kBandWarps * 32) band_trace_kernel(BandDev D, const long long* toff,
                                                                     const long long* moff, double* M) {
  extern __shared__ double band_sm[];
  __shared__ int item_s;
  constexpr int NC = kBandCols, NW = kBandWarps, RA = kRowsAhead;
  double* part = band_sm;                       // NW x NC partial row sums
  double* xs = part + NW * NC;                  // NC
  double* ring = xs + NC;                       // W x NC: the last W rows of the sweep
  double* rows = ring + (D.max_w + 1) * NC;     // RA row buffers
  const int RS = D.max_w + 2 + NC;              // row buffer stride
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  double* Z = D.Z + (long long)blockIdx.x * D.max_n * NC;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(D.flags + 1, 1);
    __syncthreads();
    const int it = item_s;
    if (it >= D.n_items) break;
    const int4 I = D.items[it];
    const int f = I.x, cnt = I.z, p0 = I.w;
    const long long o = D.off[f], t0 = toff[f];
    const int n = (int)(D.off[f + 1] - o), w = D.w[f], W = w + 1;
    const long long tf = toff[f + 1] - t0;
    const double* L = D.L + D.boff[f];
    const double* dinv = D.dinv + o;
    const int col_b = lane < cnt ? D.tcol[t0 + I.y + lane] : -1;
    const int col_p = lane < cnt ? D.tpos[t0 + I.y + lane] : -1;
    // copy row `row` of the factor (and its pivot reciprocal; with zrow, the
    // forward values of row - W) into its buffer; one commit group per call
    auto fetch = [&](int row, bool zrow) {
      if (row >= p0 && row < n) {
        double* dst = rows + (row % RA) * RS;
        const double* src = L + (long long)row * W;
        for (int e = threadIdx.x; e < W; e += blockDim.x) cp_async8(dst + e, src + e);
        if (threadIdx.x == 0) cp_async8(dst + W, dinv + row);
        if (zrow && row - W >= p0 && threadIdx.x < NC)
          cp_async8(dst + W + 1 + threadIdx.x, Z + (long long)(row - W) * NC + threadIdx.x);
      }
      cp_async_commit();
    };
    for (int e = threadIdx.x; e < W * NC; e += blockDim.x) ring[e] = 0.0;
    // forward: L y = e_b from row p0 on
    for (int q = 0; q < RA - 1; ++q) fetch(p0 + q, false);
    cp_async_wait<RA - 2>();
    __syncthreads();
    for (int i = p0; i < n; ++i) {
      fetch(i + RA - 1, false);  // into the buffer row i-1 has left
      const double* Li = rows + (i % RA) * RS + w;  // Li[-k] = L(i, i-k), Li[1] = 1/L(i,i)
      const int kmax = min(w, i - p0);
      double acc = 0.0;
      if (1 + g <= kmax) {
        int sl = (i - 1 - g) % W;
        for (int k = 1 + g; k <= kmax; k += NW) {
          acc = fma(Li[-k], ring[sl * NC + lane], acc);
          sl -= NW;
          while (sl < 0) sl += W;
        }
      }
      part[g * NC + lane] = acc;
      __syncthreads();
      if (g == 0) {
        double s = 0.0;
        for (int q = 0; q < NW; ++q) s += part[q * NC + lane];
        const double y = ((i == col_p ? 1.0 : 0.0) - s) * Li[1];
        ring[(i % W) * NC + lane] = y;
        Z[(long long)i * NC + lane] = y;
      }
      cp_async_wait<RA - 2>();  // row i + 1 is in
      __syncthreads();
    }
    // all forward values are written before the backward sweep copies them
    __threadfence_block();
    // backward: L^T x = y; slot of row t holds y_t minus the rows applied so far
    for (int e = threadIdx.x; e < W * NC; e += blockDim.x) {
      const int rr = n - 1 - e / NC, ln = e % NC;
      if (rr >= 0) ring[(rr % W) * NC + ln] = rr >= p0 ? Z[(long long)rr * NC + ln] : 0.0;
    }
    for (int q = 0; q < RA - 1; ++q) fetch(n - 1 - q, true);
    cp_async_wait<RA - 2>();
    __syncthreads();
    const int* tat = D.trace_at + o;
    double* Mf = M + moff[f];
    // x is needed at rows >= p0 only: an entry M_f[a][b] with a above the
    // item's first column is the mirror of one that column a's item computes
    for (int t = n - 1; t >= p0; --t) {
      fetch(t - RA + 1, true);
      const double* Lt = rows + (t % RA) * RS + w;  // Lt[1] = 1/L(t,t), Lt[2 + lane] = y(t - W)
      if (g == 0) {
        const int st = (t % W) * NC + lane;
        const double x = ring[st] * Lt[1];
        xs[lane] = x;
        const int a = tat[t];
        if (a >= 0 && col_b >= 0) Mf[(long long)a * tf + col_b] = x;
        ring[st] = t - W >= p0 ? Lt[2 + lane] : 0.0;  // the row that takes this slot next
      }
      __syncthreads();
      const double x = xs[lane];
      const int kmax = min(w, t - p0);
      if (1 + g <= kmax) {
        int sl = (t - 1 - g) % W;
        for (int k = 1 + g; k <= kmax; k += NW) {
          double* q = ring + sl * NC + lane;
          *q = fma(-Lt[-k], x, *q);
          sl -= NW;
          while (sl < 0) sl += W;
        }
      }
      cp_async_wait<RA - 2>();  // row t - 1 is in
      __syncthreads();
    }
  }
  cp_async_wait<0>();
}

// Of each mirrored pair M_f[a][b], M_f[b][a], the entry in the column of
// the trace node further up the ordering is computed by every item (the
// row lies below that column's first position); copy it onto the other.
__global__ void band_symmetrize_kernel(int nf, const long long* toff, const long long* moff, const int* tposa,
                                       double* M) {
  const long long total = moff[nf];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int f = fracture_of(moff, nf, e);
    const long long t = toff[f + 1] - toff[f], loc = e - moff[f];
    const long long a = loc / t, b = loc % t;
    if (a >= b) continue;
    double* Mf = M + moff[f];
    if (tposa[toff[f] + a] < tposa[toff[f] + b])
      Mf[a * t + b] = Mf[b * t + a];
    else
      Mf[b * t + a] = Mf[a * t + b];
  }
}

// z[offset[f] + position] = v[offset[f] + node at that position]
__global__ void band_gather_kernel(BandDev D, int n_h, const double* __restrict__ v, double* __restrict__ z) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_h;
       r += (long long)gridDim.x * blockDim.x) {
    const int f = fracture_of(D.off, D.n_f, r);
    const long long o = D.off[f];
    z[r] = v[o + D.perm[r]];
  }
}

// One warp per fracture; z holds the permuted right-hand side on entry and
// the forward values on exit; y receives A_f^{-1} v in the caller's order.
__global__ void band_solve_kernel(BandDev D, double* z, double* y) {
  extern __shared__ double band_sm[];
  constexpr int RA = kRowsAhead;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  if (gw >= D.n_f) return;  // whole warps only: no block barrier below
  const int f = D.order[gw];
  const long long o = D.off[f];
  const int n = (int)(D.off[f + 1] - o), w = D.w[f], W = w + 1;
  const double* L = D.L + D.boff[f];
  const double* dinv = D.dinv + o;
  const int* perm = D.perm + o;
  const int RS = D.max_w + 3;
  double* ring = band_sm + (long long)wib * ((D.max_w + 1) + RA * RS);
  double* rows = ring + (D.max_w + 1);
  double* zf = z + o;
  // row buffer: L(row, row-w..row), 1/L(row,row), and z[row] (forward) or
  // z[row - W] (backward)
  auto fetch = [&](int row, int zoff) {
    if (row >= 0 && row < n) {
      double* dst = rows + (row % RA) * RS;
      const double* src = L + (long long)row * W;
      for (int e = lane; e < W; e += 32) cp_async8(dst + e, src + e);
      if (lane == 0) cp_async8(dst + W, dinv + row);
      if (lane == 1 && row - zoff >= 0) cp_async8(dst + W + 1, zf + row - zoff);
    }
    cp_async_commit();
  };
  for (int q = 0; q < RA - 1; ++q) fetch(q, 0);
  cp_async_wait<RA - 2>();
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    fetch(i + RA - 1, 0);
    const double* Li = rows + (i % RA) * RS + w;  // Li[1] = 1/L(i,i), Li[2] = z[i]
    const int kmax = min(w, i);
    double acc = 0.0;
    for (int k = 1 + lane; k <= kmax; k += 32) acc = fma(Li[-k], ring[(i - k) % W], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
      const double yi = (Li[2] - acc) * Li[1];
      ring[i % W] = yi;
      zf[i] = yi;
    }
    cp_async_wait<RA - 2>();
    __syncwarp();
  }
  __threadfence_block();
  for (int e = lane; e < W; e += 32) {
    const int rr = n - 1 - e;
    if (rr >= 0) ring[rr % W] = zf[rr];
  }
  for (int q = 0; q < RA - 1; ++q) fetch(n - 1 - q, W);
  cp_async_wait<RA - 2>();
  __syncwarp();
  for (int t = n - 1; t >= 0; --t) {
    fetch(t - RA + 1, W);
    const double* Lt = rows + (t % RA) * RS + w;  // Lt[1] = 1/L(t,t), Lt[2] = z[t - W]
    const double x = ring[t % W] * Lt[1];
    __syncwarp();
    if (lane == 0) {
      y[o + perm[t]] = x;
      ring[t % W] = t - W >= 0 ? Lt[2] : 0.0;
    }
    const int kmax = min(w, t);
    for (int k = 1 + lane; k <= kmax; k += 32) {
      const int sl = (t - k) % W;
      ring[sl] = fma(-Lt[-k], x, ring[sl]);
    }
    cp_async_wait<RA - 2>();
    __syncwarp();
  }
  cp_async_wait<0>();
}

int grid_for(long long work, int block) {
  const long long g = (work + block - 1) / block;
  return (int)std::max(1LL, std::min<long long>(g, 16LL * num_sms()));
}

cudaError_t allow_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Reverse Cuthill-McKee (Cuthill & McKee 1969; reversed as in George 1971)
// from pseudo-peripheral roots (George & Liu 1979), one connected component
// at a time; neighbours are visited by increasing degree, ties by index.
// Returns order[position] = local node.
std::vector<int> rcm_order(int n, const std::vector<int>& aptr, const std::vector<int>& adj) {
  std::vector<int> order, queue(n), dist(n, 0), stamp(n, -1), nbr;
  std::vector<char> placed(n, 0);
  order.reserve(n);
  auto deg = [&](int v) { return aptr[v + 1] - aptr[v]; };
  int round = 0;
  auto bfs = [&](int root) {  // over unplaced nodes; returns the visit count
    ++round;
    int head = 0, tail = 0;
    queue[tail++] = root;
    stamp[root] = round;
    dist[root] = 0;
    while (head < tail) {
      const int v = queue[head++];
      for (int p = aptr[v]; p < aptr[v + 1]; ++p) {
        const int u = adj[p];
        if (placed[u] || stamp[u] == round) continue;
        stamp[u] = round;
        dist[u] = dist[v] + 1;
        queue[tail++] = u;
      }
    }
    return tail;
  };
  for (int s = 0; s < n; ++s) {
    if (placed[s]) continue;
    int root = s, depth = -1;
    for (int it = 0; it < 16; ++it) {
      const int cnt = bfs(root);
      const int d = dist[queue[cnt - 1]];
      if (d <= depth) break;
      depth = d;
      int best = queue[cnt - 1];
      for (int q = cnt - 1; q >= 0 && dist[queue[q]] == d; --q)
        if (deg(queue[q]) < deg(best) || (deg(queue[q]) == deg(best) && queue[q] < best)) best = queue[q];
      root = best;
    }
    size_t head = order.size();
    order.push_back(root);
    placed[root] = 1;
    while (head < order.size()) {
      const int v = order[head++];
      nbr.clear();
      for (int p = aptr[v]; p < aptr[v + 1]; ++p) {
        const int u = adj[p];
        if (!placed[u]) {
          placed[u] = 1;
          nbr.push_back(u);
        }
      }
      std::sort(nbr.begin(), nbr.end(), [&](int x, int y) { return deg(x) != deg(y) ? deg(x) < deg(y) : x < y; });
      order.insert(order.end(), nbr.begin(), nbr.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

}  // namespace

size_t band_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = 227 * 1024;
  }
  return (size_t)v;
}

int band_plan(int n_f, int n_h, const long long* offset, const std::vector<int>& rp, const std::vector<int>& col,
              const std::vector<double>& val, const std::vector<long long>& toff, const std::vector<int>& tnode,
              BandHost& H, std::string& err) {
  H = BandHost();
  H.n_f = n_f;
  H.w.assign(n_f, 0);
  H.rcm.assign(n_f, 0);
  H.boff.assign(n_f + 1, 0);
  H.gwoff.assign(n_f, -1);
  H.pos.assign(n_h, 0);
  H.perm.assign(n_h, 0);
  H.trace_at.assign(n_h, -1);
  const size_t optin = band_smem_optin();
  std::vector<int> aptr, adj, seen(n_h, -1);
  std::vector<double> work(n_f, 0.0);
  for (int f = 0; f < n_f; ++f) {
    const long long o = offset[f];
    const int n = (int)(offset[f + 1] - o);
    aptr.assign(n + 1, 0);
    adj.clear();
    for (int i = 0; i < n; ++i) {
      const long long r = o + i;
      bool diag = false;
      for (int p = rp[r]; p < rp[r + 1]; ++p) {
        const long long c = col[p];
        if (c < o || c >= o + n) {
          err = "A is not block diagonal: row " + std::to_string(r) + " of fracture " + std::to_string(f) +
                " has column " + std::to_string(c);
          return PP_EINVAL;
        }
        if (seen[c] == (int)r) {
          err = "A has a repeated entry (" + std::to_string(r) + ", " + std::to_string(c) + ")";
          return PP_EINVAL;
        }
        seen[c] = (int)r;
        if (c == r) {
          if (!(val[p] > 0.0)) {
            err = "A is not positive definite: diagonal " + std::to_string(r) + " is not positive";
            return PP_EBREAKDOWN;
          }
          diag = true;
          continue;
        }
        // the mirrored entry must exist with the same value
        bool sym = false;
        for (int q = rp[c]; q < rp[c + 1]; ++q)
          if (col[q] == r) {
            sym = val[q] == val[p];
            break;
          }
        if (!sym) {
          err = "A is not symmetric at (" + std::to_string(r) + ", " + std::to_string(c) + ")";
          return PP_EINVAL;
        }
        adj.push_back((int)(c - o));
      }
      if (!diag) {
        err = "A has no diagonal entry in row " + std::to_string(r);
        return PP_EINVAL;
      }
      aptr[i + 1] = (int)adj.size();
    }
    int w_nat = 0;
    for (int i = 0; i < n; ++i)
      for (int p = aptr[i]; p < aptr[i + 1]; ++p) w_nat = std::max(w_nat, std::abs(adj[p] - i));
    std::vector<int> ord = rcm_order(n, aptr, adj), inv(n);
    for (int p = 0; p < n; ++p) inv[ord[p]] = p;
    int w_rcm = 0;
    for (int i = 0; i < n; ++i)
      for (int p = aptr[i]; p < aptr[i + 1]; ++p) w_rcm = std::max(w_rcm, std::abs(inv[adj[p]] - inv[i]));
    const bool use_rcm = w_rcm < w_nat;
    H.rcm_used += use_rcm ? 1 : 0;
    H.rcm[f] = use_rcm ? 1 : 0;
    const int w = use_rcm ? w_rcm : w_nat;
    if (w > kBandMaxW) {
      err = "fracture " + std::to_string(f) + ": half-bandwidth " + std::to_string(w) +
            " after reordering is above " + std::to_string(kBandMaxW);
      return PP_EUNSUPPORTED;
    }
    for (int p = 0; p < n; ++p) {
      const int node = use_rcm ? ord[p] : p;
      H.perm[o + p] = node;
      H.pos[o + node] = p;
    }
    const int W = w + 1;
    H.w[f] = w;
    H.boff[f + 1] = H.boff[f] + (long long)n * W;
    const size_t win_bytes = (size_t)factor_window_doubles(W) * sizeof(double);
    if (win_bytes > optin) {
      H.gwoff[f] = H.gwin_elems;
      H.gwin_elems += factor_window_doubles(W);
    } else {
      H.factor_smem = std::max(H.factor_smem, win_bytes);
    }
    H.max_w = std::max(H.max_w, w);
    H.max_n = std::max(H.max_n, n);
    work[f] = (double)n * W * W;
  }
  H.elems = H.boff[n_f];
  H.order.resize(n_f);
  std::iota(H.order.begin(), H.order.end(), 0);
  std::stable_sort(H.order.begin(), H.order.end(), [&](int a, int b) { return work[a] > work[b]; });
  // trace columns of each fracture by position, in items of kBandCols
  const int n_T = (int)tnode.size();
  H.tcol.assign(std::max(n_T, 1), 0);
  H.tpos.assign(std::max(n_T, 1), 0);
  H.tposa.assign(std::max(n_T, 1), 0);
  std::vector<std::pair<int, int>> slots;
  std::vector<double> cost;
  for (int f = 0; f < n_f; ++f) {
    const long long t0 = toff[f], t1 = toff[f + 1], o = offset[f];
    const int n = (int)(offset[f + 1] - o);
    slots.clear();
    for (long long a = 0; a < t1 - t0; ++a) {
      const int node = tnode[t0 + a];
      const int p = H.pos[node];
      H.trace_at[o + p] = (int)a;
      slots.push_back({p, (int)a});
    }
    std::sort(slots.begin(), slots.end());
    for (size_t s = 0; s < slots.size(); ++s) {
      H.tpos[t0 + s] = slots[s].first;
      H.tcol[t0 + s] = slots[s].second;
      H.tposa[t0 + slots[s].second] = slots[s].first;
    }
    for (size_t s0 = 0; s0 < slots.size(); s0 += kBandCols) {
      const int cnt = (int)std::min<size_t>(kBandCols, slots.size() - s0);
      H.items.push_back(make_int4(f, (int)s0, cnt, slots[s0].first));
      cost.push_back((double)(n - slots[s0].first) * (H.w[f] + 1));
    }
  }
  std::vector<int> idx(H.items.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int4> sorted(H.items.size());
  for (size_t i = 0; i < idx.size(); ++i) sorted[i] = H.items[idx[i]];
  H.items.swap(sorted);
  H.n_items = (int)H.items.size();
  return PP_OK;
}

cudaError_t band_fill(const BandDev& D, int n_h, const int* rp, const int* col, const double* val, cudaStream_t s) {
  band_fill_kernel<<<grid_for(n_h, 256), 256, 0, s>>>(D, n_h, rp, col, val);
  return cudaGetLastError();
}

cudaError_t band_factor(const BandDev& D, cudaStream_t s) {
  cudaError_t e = allow_smem((const void*)band_factor_kernel, D.factor_smem);
  if (e != cudaSuccess) return e;
  band_factor_kernel<<<D.n_f, kFactorThreads, D.factor_smem, s>>>(D);
  return cudaGetLastError();
}

cudaError_t band_trace_blocks(const BandDev& D, const long long* toff, const long long* moff, double* M,
                              cudaStream_t s) {
  if (D.n_items > 0) {
    const size_t sm = sizeof(double) * trace_smem_doubles(D.max_w);
    cudaError_t e = allow_smem((const void*)band_trace_kernel, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.flags + 1, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    band_trace_kernel<<<D.grid_trace, kBandWarps * 32, sm, s>>>(D, toff, moff, M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  band_symmetrize_kernel<<<8 * num_sms(), 256, 0, s>>>(D.n_f, toff, moff, D.tposa, M);
  return cudaGetLastError();
}

cudaError_t band_solve(const BandDev& D, int n_h, const double* v, double* y, double* z, cudaStream_t s) {
  constexpr int kWarps = 4;
  const size_t sm = sizeof(double) * kWarps * ((size_t)(D.max_w + 1) + kRowsAhead * (size_t)(D.max_w + 3));
  cudaError_t e = allow_smem((const void*)band_solve_kernel, sm);
  if (e != cudaSuccess) return e;
  band_gather_kernel<<<grid_for(n_h, 256), 256, 0, s>>>(D, n_h, v, z);
  band_solve_kernel<<<(D.n_f + kWarps - 1) / kWarps, kWarps * 32, sm, s>>>(D, z, y);
  return cudaGetLastError();
}

}  // namespace pp

extern "C" int pp_fracture_bands(int n_f, const long long* offset, const int* rowptr, const int* col,
                                 const double* val, int* w_out, int* rcm_out) {
  using namespace pp;
  if (n_f <= 0 || !offset || !rowptr || !w_out) return fail(nullptr, PP_EINVAL, "NULL argument or n_f <= 0");
  if (offset[0] != 0) return fail(nullptr, PP_EINVAL, "offset[0] must be 0");
  for (int f = 0; f < n_f; ++f)
    if (offset[f + 1] <= offset[f]) return fail(nullptr, PP_EINVAL, "fracture " + std::to_string(f) + " has no nodes");
  const long long n_h = offset[n_f];
  if (n_h > INT_MAX) return fail(nullptr, PP_EINVAL, "too many nodes");
  const long long nnz = rowptr[n_h];
  if (rowptr[0] != 0 || nnz < 0 || (nnz > 0 && (!col || !val))) return fail(nullptr, PP_EINVAL, "bad CSR arrays");
  std::vector<int> rp(rowptr, rowptr + n_h + 1), cc(col, col + nnz);
  std::vector<double> vv(val, val + nnz);
  for (long long r = 0; r < n_h; ++r)
    if (rp[r + 1] < rp[r]) return fail(nullptr, PP_EINVAL, "rowptr is not monotone");
  for (long long p = 0; p < nnz; ++p)
    if (cc[p] < 0 || cc[p] >= n_h) return fail(nullptr, PP_EINVAL, "A column out of range");
  BandHost H;
  std::string err;
  const std::vector<long long> toff(n_f + 1, 0);
  const std::vector<int> tnode;
  const int rc = band_plan(n_f, (int)n_h, offset, rp, cc, vv, toff, tnode, H, err);
  if (rc) return fail(nullptr, rc, err);
  for (int f = 0; f < n_f; ++f) {
    w_out[f] = H.w[f];
    if (rcm_out) rcm_out[f] = H.rcm[f];
  }
  return PP_OK;
}
