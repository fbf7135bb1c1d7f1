// Device-side building blocks shared by the kernels: operator tables, tile geometry,
// shared-memory tile staging, block / grid reductions and a capped grid barrier.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace dgk {

// Flags a device-side solve may raise (OR-ed into the status word).
enum : int { kFlagNoconv = 1, kFlagTimeout = 2, kFlagBreakdown = 4, kFlagNonfinite = 8 };

// A 1D block-tridiagonal periodic operator whose neighbour blocks are rank one:
//   (Op u)_c = M u_c + a (r . u_{c+1}) + d (s . u_{c-1})
// Instances: the central-flux derivative (Sec. 4.2, Eq. discrete_der: M = C0/h,
// a = muR/h, r = lL, d = -muL/h, s = lR), the symmetrically scaled LDG stiffness and the
// dG Laplacian (Sec. 6).
template <typename T, int N>
struct Op1D {
  T M[N][N];
  T a[N], r[N], d[N], s[N];
  // the first cell of a line at a Dirichlet boundary (LDG operators; the derivatives keep the
  // periodic values and handle the boundary through ghost traces): own block, lift of the
  // right neighbour's trace, and the vector of its own trace seen by the second cell
  T Mf[N][N];
  T af[N], sf[N];
};

template <typename T, int N>
struct Ops2D {
  Op1D<T, N> dx, dy;  // central-flux derivatives d/dx, d/dy
  Op1D<T, N> kx, ky;  // W^-1/2 A W^-1/2 = I (x) kx + ky (x) I   (CG operator)
  Op1D<T, N> lx, ly;  // -Delta_h = W^-1 A = lx + ly
  T sw[N * N];        // sqrt(W_ab) per node of a cell
  T isw[N * N];       // 1 / sqrt(W_ab)
  T wq[N * N];        // W_ab = (hy w_a / 2)(hx w_b / 2)
};

// The CG operator alone, for the compensated (double-float) operator apply of the float32
// inner solve.
template <typename T, int N>
struct OpsK {
  Op1D<T, N> kx, ky;
};

struct Geom {
  int Nx, Ny;          // cells
  int TX, TY;          // tile (cells)
  int tilesX, tilesY;
  int bc;              // 0: periodic, 1: homogeneous Dirichlet (zero outside the domain)
};

// One tile of cells and its one-cell halo ring in shared memory: box cell (br, bc) holds
// grid cell (ty0 + br - 1, tx0 + bc - 1) (periodic wrap); the box row stride is BW = TX + 2.
// A staged cell occupies N*N + 1 values (one pad value: with a stride of N*N, a multiple of
// the 32 banks for most N, the lanes of a warp reading the same node of different cells or
// lines would hit the same bank).
struct TileBox {
  int ty0, tx0, TYe, TXe, BW;
  unsigned mTXe;  // magic_of(TXe): cell c of the tile is in tile row quot(c, mTXe)
};

// Integer quotients by a divisor d that is fixed for a loop: m = magic_of(d) (once), then
// quot(c, m) = c / d for 0 <= c with c * d < 2^32 (one multiply-high in place of a division).
// With m = floor((2^32 - 1) / d) + 1 = (2^32 + e) / d, 0 <= e < d, the product c m / 2^32 is
// c / d + c e / (d 2^32), and c e < 2^32 keeps the added part below 1/d, so its floor is the
// quotient.  d = 1 (m would be 2^32) is encoded as m = 0.
__host__ __device__ __forceinline__ unsigned magic_of(int d) { return d == 1 ? 0u : 0xFFFFFFFFu / unsigned(d) + 1u; }
__device__ __forceinline__ int quot(int c, unsigned m) { return m ? int(__umulhi(unsigned(c), m)) : c; }

__device__ __forceinline__ int wrap_index(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

__device__ __forceinline__ TileBox make_box(const Geom& G, int tile) {
  TileBox B;
  const int tyi = tile / G.tilesX, txi = tile - (tile / G.tilesX) * G.tilesX;
  B.ty0 = tyi * G.TY;
  B.tx0 = txi * G.TX;
  B.TYe = min(G.TY, G.Ny - B.ty0);
  B.TXe = min(G.TX, G.Nx - B.tx0);
  B.BW = G.TX + 2;
  B.mTXe = magic_of(B.TXe);
  return B;
}

// Stage a field into the box: load(g, k, interior) returns the value of node k of the cell
// at global offset g (k = a*N + b).  With corners == false the four corner cells are skipped
// (the 5-cell operators never read them).
template <typename T, int N, class LoadF>
__device__ __forceinline__ void stage_box(const Geom& G, const TileBox& B, T* sU, bool corners, LoadF&& load) {
  constexpr int NN = N * N;
  const int BWe = B.TXe + 2, BHe = B.TYe + 2;
  const int rowlen = BWe * NN;
  const int total = BHe * rowlen;
  const unsigned mrow = magic_of(rowlen);
  // one flat loop over the whole box, so that a thread's loads of several rows are in flight
  // together
#pragma unroll 4
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int br = quot(i, mrow);
    const int j = i - br * rowlen;
    const int bc = j / NN;
    const int k = j - bc * NN;
    const bool rowhalo = (br == 0) || (br == BHe - 1);
    const bool colhalo = (bc == 0) || (bc == BWe - 1);
    if (rowhalo && colhalo && !corners) continue;
    const int gy = B.ty0 + br - 1, gx = B.tx0 + bc - 1;
    if (G.bc && (gy < 0 || gy >= G.Ny || gx < 0 || gx >= G.Nx)) {  // Dirichlet: zero outside
      sU[(br * B.BW + bc) * (NN + 1) + k] = T(0);
      continue;
    }
    const int cy = wrap_index(gy, G.Ny);
    const int cx = wrap_index(gx, G.Nx);
    const size_t g = ((size_t)cy * G.Nx + cx) * NN + k;
    sU[(br * B.BW + bc) * (NN + 1) + k] = load(g, k, !(rowhalo || colhalo));
  }
}

// Face traces of every line of the cells an operator application needs (x-lines read from
// sUx, y-lines from sUy, which may be the same array):
//   x-lines (rows a) of cells ry in [0, TYe), rx in [-1, TXe]:  tXR = ox.r . row, tXL = ox.s . row
//   y-lines (cols b) of cells ry in [-1, TYe], rx in [0, TXe):   tYR = oy.r . col, tYL = oy.s . col
// With full == true the x-lines also cover the halo rows and the y-lines the halo columns.
template <typename T, int N>
__device__ __forceinline__ void line_traces(const TileBox& B, const T* sUx, const T* sUy,
                                            const Op1D<T, N>& ox, const Op1D<T, N>& oy, T* tXR,
                                            T* tXL, T* tYR, T* tYL, bool full) {
  constexpr int NN = N * N;
  const int y0 = full ? -1 : 0, y1 = full ? B.TYe + 1 : B.TYe;
  const int x0 = full ? -1 : 0, x1 = full ? B.TXe + 1 : B.TXe;
  const int wx = B.TXe + 2, hx = y1 - y0;   // x-line cells: rows y0..y1-1, cols -1..TXe
  const int wy = x1 - x0, hy = B.TYe + 2;   // y-line cells: rows -1..TYe, cols x0..x1-1
  const int nx = hx * wx * N, ny = hy * wy * N;
  const unsigned mwx = magic_of(wx), mwy = magic_of(wy);
  // the trace coefficients: in registers for float32 (for float64 the registers are scarcer
  // than the shared-memory issue slots of this FMA-bound path)
  T xr[N], xs[N], yr[N], ys[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if constexpr (sizeof(T) == 4) {
      xr[j] = ox.r[j];
      xs[j] = ox.s[j];
      yr[j] = oy.r[j];
      ys[j] = oy.s[j];
    }
  }
  for (int i = threadIdx.x; i < nx + ny; i += blockDim.x) {
    if (i < nx) {
      const int c = i / N, line = i - (i / N) * N;
      const int cq = quot(c, mwx);
      const int ry = cq + y0, rx = c - cq * wx - 1;
      const int lc = (ry + 1) * B.BW + rx + 1;
      const T* u = sUx + lc * (NN + 1) + line * N;
      T tr = T(0), tl = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if constexpr (sizeof(T) == 4) {
          tr = fma(xr[j], u[j], tr);
          tl = fma(xs[j], u[j], tl);
        } else {
          tr = fma(ox.r[j], u[j], tr);
          tl = fma(ox.s[j], u[j], tl);
        }
      }
      tXR[lc * N + line] = tr;
      tXL[lc * N + line] = tl;
    } else {
      const int ii = i - nx;
      const int c = ii / N, line = ii - (ii / N) * N;
      const int cq = quot(c, mwy);
      const int ry = cq - 1, rx = c - cq * wy + x0;
      const int lc = (ry + 1) * B.BW + rx + 1;
      const T* u = sUy + lc * (NN + 1) + line;
      T tr = T(0), tl = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if constexpr (sizeof(T) == 4) {
          tr = fma(yr[j], u[j * N], tr);
          tl = fma(ys[j], u[j * N], tl);
        } else {
          tr = fma(oy.r[j], u[j * N], tr);
          tl = fma(oy.s[j], u[j * N], tl);
        }
      }
      tYR[lc * N + line] = tr;
      tYL[lc * N + line] = tl;
    }
  }
}

// (Op_x u) at node (a, b) of box cell lc, using the staged field and its x-line traces; first:
// the cell is the first of its line at a Dirichlet boundary (own block Mf).
template <typename T, int N>
__device__ __forceinline__ T op_x_at(const T* sU, const T* tXR, const T* tXL, const Op1D<T, N>& o,
                                     int lc, int a, int b, bool first = false) {
  const T* u = sU + lc * (N * N + 1) + a * N;
  const T* Mrow = first ? o.Mf[b] : o.M[b];
  T acc = (first ? o.af[b] : o.a[b]) * tXR[(lc + 1) * N + a];
  acc = fma(o.d[b], tXL[(lc - 1) * N + a], acc);
#pragma unroll
  for (int j = 0; j < N; ++j) acc = fma(Mrow[j], u[j], acc);
  return acc;
}

// (Op_y u) at node (a, b) of box cell lc (the c+1 neighbour in y is one box row up).
template <typename T, int N>
__device__ __forceinline__ T op_y_at(const T* sU, const T* tYR, const T* tYL, const Op1D<T, N>& o,
                                     int lc, int BW, int a, int b, bool first = false) {
  const T* u = sU + lc * (N * N + 1) + b;
  const T* Mrow = first ? o.Mf[a] : o.M[a];
  T acc = (first ? o.af[a] : o.a[a]) * tYR[(lc + BW) * N + b];
  acc = fma(o.d[a], tYL[(lc - BW) * N + b], acc);
#pragma unroll
  for (int j = 0; j < N; ++j) acc = fma(Mrow[j], u[j * N], acc);
  return acc;
}

// Homogeneous Dirichlet boundaries for the LDG operators: the trace that the second cell of a
// line sees of the first one uses the first cell's own vector sf (line_traces wrote s . u).
// Run after line_traces (and a block synchronisation) on Dirichlet grids only.
template <typename T, int N>
__device__ __forceinline__ void dirichlet_first_traces(const TileBox& B, const T* sUx, const T* sUy,
                                                       const Op1D<T, N>& ox, const Op1D<T, N>& oy, T* tXL, T* tYL) {
  constexpr int NN = N * N;
  const int nx = B.tx0 == 0 ? B.TYe * N : 0;   // x-lines of the tile's first column
  const int ny = B.ty0 == 0 ? B.TXe * N : 0;   // y-lines of the tile's first row
  for (int i = threadIdx.x; i < nx + ny; i += blockDim.x) {
    if (i < nx) {
      const int ry = i / N, line = i - (i / N) * N;
      const int lc = (ry + 1) * B.BW + 1;
      const T* u = sUx + lc * (NN + 1) + line * N;
      T tl = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) tl = fma(ox.sf[j], u[j], tl);
      tXL[lc * N + line] = tl;
    } else {
      const int ii = i - nx;
      const int rx = ii / N, line = ii - (ii / N) * N;
      const int lc = B.BW + rx + 1;
      const T* u = sUy + lc * (NN + 1) + line;
      T tl = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) tl = fma(oy.sf[j], u[j * N], tl);
      tYL[lc * N + line] = tl;
    }
  }
}

// Homogeneous Dirichlet boundaries for the central-flux derivative (Sec. 3: the flux on a
// boundary face is the boundary value, f^ = 0): the ghost cell beyond a boundary face gets the
// negated trace of the boundary cell on that face, so that the average flux there vanishes.
// Overwrites the traces of the ghost cells of the tile's lines (x-lines of rows [y0, y1),
// y-lines of columns [x0, x1), as line_traces computed them with the same `full`).
template <typename T, int N>
__device__ __forceinline__ void dirichlet_ghost_traces(const Geom& G, const TileBox& B, T* tXR, T* tXL, T* tYR,
                                                       T* tYL, bool full) {
  const int y0 = full ? -1 : 0, y1 = full ? B.TYe + 1 : B.TYe;
  const int x0 = full ? -1 : 0, x1 = full ? B.TXe + 1 : B.TXe;
  const bool left = B.tx0 == 0, right = B.tx0 + B.TXe == G.Nx;
  const bool bottom = B.ty0 == 0, top = B.ty0 + B.TYe == G.Ny;
  const int nx = (y1 - y0) * N, ny = (x1 - x0) * N;
  for (int i = threadIdx.x; i < nx + ny; i += blockDim.x) {
    if (i < nx) {
      const int ry = i / N + y0, line = i - (i / N) * N;
      const int row = (ry + 1) * B.BW;
      if (left) tXL[(row + 0) * N + line] = -tXR[(row + 1) * N + line];
      if (right) tXR[(row + B.TXe + 1) * N + line] = -tXL[(row + B.TXe) * N + line];
    } else {
      const int ii = i - nx;
      const int rx = ii / N + x0, line = ii - (ii / N) * N;
      const int col = rx + 1;
      if (bottom) tYL[(0 * B.BW + col) * N + line] = -tYR[(1 * B.BW + col) * N + line];
      if (top) tYR[((B.TYe + 1) * B.BW + col) * N + line] = -tYL[(B.TYe * B.BW + col) * N + line];
    }
  }
}

// ---- grid-stride passes --------------------------------------------------------------------

// A grid-stride loop over [first, n) in rounds of U strides: the loads of a round (ld(i)) are
// all issued before its uses (use(i, value), in increasing i, so sums accumulate in the same
// order as a plain loop).  With one load in flight per thread, the 16-32 resident warps of an
// SM reach a fraction of the HBM bandwidth; U loads in flight multiply it.
template <int U, class Ld, class Use>
__device__ __forceinline__ void strided_pass(size_t first, size_t n, size_t stride, Ld&& ld, Use&& use) {
  using V = decltype(ld(size_t(0)));
  for (size_t i0 = first; i0 < n; i0 += U * stride) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t i = i0 + u * stride;
      if (i < n) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t i = i0 + u * stride;
      if (i < n) use(i, v[u]);
    }
  }
}

// ---- reductions ------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum_down(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum; the result is valid in thread 0.  red: >= 32 values of scratch.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum_down(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T t = T(0);
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? red[l] : T(0);
    t = warp_sum_down(t);
  }
  return t;
}

// Sum of G per-block partials p[i*stride], in a fixed order, returned to every thread of a
// one-warp launch.  Reads bypass L1 (written by other blocks).
template <typename T>
__device__ __forceinline__ T sum_partials(const T* p, int G, int stride, T* bcast) {
  if (threadIdx.x < 32) {
    T v = T(0);
    for (int i = threadIdx.x; i < G; i += 32) v += __ldcg(p + (size_t)i * stride);
    v = warp_sum_down(v);
    if (threadIdx.x == 0) *bcast = v;
  }
  __syncthreads();
  const T r = *bcast;
  __syncthreads();
  return r;
}

// The same with the whole block: thread t adds the partials t, t + blockDim.x, ... in
// order, then a fixed-shape block reduction.  Every block computes the bit-identical value
// (the order depends only on G and blockDim.x); one round of loads instead of G / 32.
template <typename T>
__device__ __forceinline__ T sum_partials_block(const T* p, int G, int stride, T* red, T* bcast) {
  T v = T(0);
  for (int i = threadIdx.x; i < G; i += blockDim.x) v += __ldcg(p + (size_t)i * stride);
  v = block_sum(v, red);
  if (threadIdx.x == 0) *bcast = v;
  __syncthreads();
  const T r = *bcast;
  __syncthreads();
  return r;
}

// ---- grid barrier for persistent cooperative kernels -----------------------------------

struct SyncState {
  unsigned int count;
  unsigned int gen;
  int error;
  unsigned int ticket;  // work-unit tickets of the dynamically scheduled phases (next_unit)
};

// Waits of a block at the barrier give up after this many polls (~1 s with the sleep
// below) and raise kFlagTimeout; every later barrier then returns false at once.
constexpr unsigned long long kSpinCap = 1ull << 23;

// The nblk blocks of a (virtual) grid meet here: all blocks of a cooperative launch, or the
// blocks of one group of a batched launch.  Returns false if any block raised an error.
__device__ __forceinline__ bool grid_barrier(SyncState* s, int* s_flag, unsigned int nblk) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &s->gen;
    volatile int* verr = &s->error;
    const unsigned int gen0 = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&s->count, 1u) + 1u;
    if (arrived == nblk) {
      atomicExch(&s->count, 0u);
      __threadfence();
      atomicAdd(&s->gen, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == gen0) {
        if (*verr) break;
        if (++spins > kSpinCap) {
          atomicCAS(&s->error, 0, kFlagTimeout);
          break;
        }
        if (spins > 4096) __nanosleep(100);  // poll tightly first: most waits are short
      }
    }
    __threadfence();
    *s_flag = *verr;
  }
  __syncthreads();
  return *s_flag == 0;
}

// All threads of all blocks of this thread-block cluster meet here: the hardware cluster
// barrier, with release / acquire ordering of memory (global included) at cluster scope.
// The blocks of a cluster are co-scheduled by construction, so the wait needs no cap.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---- lines of a 2D DFT in shared memory ---------------------------------------------------

template <typename T>
struct Cplx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
  return Cplx<T>{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}

// In-place DFT of one line of length L held in shared memory s[0..L), computed by the
// whole block.  tw[m] = exp(-2 pi i m / L), m < L (host-computed).  inverse: conjugate
// twiddles (no 1/L factor).  Power-of-two L: iterative radix-2 decimation in time on
// bit-reversed input (the caller loads s[bitrev(j)] = x[j]), two stages per pass;
// otherwise a direct O(L^2) sum into tmp[0..L) copied back.
template <typename T>
__device__ __forceinline__ void dft_line(Cplx<T>* s, Cplx<T>* tmp, int L, int log2L, const Cplx<T>* tw,
                                         bool inverse) {
  if (log2L >= 0) {
    int half = 1;
    if (log2L & 1) {  // an odd number of stages: one radix-2 stage first
      for (int t = threadIdx.x; t < L / 2; t += blockDim.x) {
        Cplx<T> w = tw[0];
        if (inverse) w.im = -w.im;
        const Cplx<T> u = s[2 * t];
        const Cplx<T> v = cmul(w, s[2 * t + 1]);
        s[2 * t] = Cplx<T>{u.re + v.re, u.im + v.im};
        s[2 * t + 1] = Cplx<T>{u.re - v.re, u.im - v.im};
      }
      __syncthreads();
      half = 2;
    }
    // two radix-2 stages (half, 2 half) per pass over groups of four: half the block
    // synchronisations of one stage per pass
    for (; half < L; half <<= 2) {
      const int s2 = L / (2 * half), s4 = L / (4 * half);
      for (int t = threadIdx.x; t < L / 4; t += blockDim.x) {
        const int grp = t / half, pos = t - grp * half;
        const int i0 = grp * 4 * half + pos;
        Cplx<T> w2 = tw[pos * s2], w4 = tw[pos * s4];
        if (inverse) {
          w2.im = -w2.im;
          w4.im = -w4.im;
        }
        const Cplx<T> a = s[i0], b = cmul(w2, s[i0 + half]);
        const Cplx<T> c = s[i0 + 2 * half], d = cmul(w2, s[i0 + 3 * half]);
        const Cplx<T> A1{a.re + b.re, a.im + b.im}, B1{a.re - b.re, a.im - b.im};
        const Cplx<T> C1 = cmul(w4, Cplx<T>{c.re + d.re, c.im + d.im});
        Cplx<T> D1 = cmul(w4, Cplx<T>{c.re - d.re, c.im - d.im});
        // the second stage's twiddle for the odd half is w4 times exp(-+ i pi / 2)
        D1 = inverse ? Cplx<T>{-D1.im, D1.re} : Cplx<T>{D1.im, -D1.re};
        s[i0] = Cplx<T>{A1.re + C1.re, A1.im + C1.im};
        s[i0 + 2 * half] = Cplx<T>{A1.re - C1.re, A1.im - C1.im};
        s[i0 + half] = Cplx<T>{B1.re + D1.re, B1.im + D1.im};
        s[i0 + 3 * half] = Cplx<T>{B1.re - D1.re, B1.im - D1.im};
      }
      __syncthreads();
    }
  } else {
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
      T re = T(0), im = T(0);
      int m = 0;  // (j * k) mod L, advanced incrementally
      for (int j = 0; j < L; ++j) {
        Cplx<T> w = tw[m];
        if (inverse) w.im = -w.im;
        const Cplx<T> v = cmul(w, s[j]);
        re += v.re;
        im += v.im;
        m += k;
        if (m >= L) m -= L;
      }
      tmp[k] = Cplx<T>{re, im};
    }
    __syncthreads();
    for (int k = threadIdx.x; k < L; k += blockDim.x) s[k] = tmp[k];
    __syncthreads();
  }
}

// Position of element j of a line in the shared buffer before dft_line.
__device__ __forceinline__ int dft_slot(int j, int log2L) {
  return log2L > 0 ? int(__brev(unsigned(j)) >> (32 - log2L)) : j;
}

template <typename T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) {
  return Cplx<T>{a.re + b.re, a.im + b.im};
}

template <typename T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) {
  return Cplx<T>{a.re - b.re, a.im - b.im};
}

// DFTs of `count` lines of length L held one after another in shared memory (line c at
// s + c L), computed by the whole block; tw, inverse and the non-power-of-two fallback (a
// direct sum into tmp[0 .. count L)) as for dft_line.  Power-of-two L: with dif == false the
// decimation-in-time form of dft_line (bit-reversed input, natural output); with dif == true
// decimation in frequency (natural input, output in bit-reversed order: element k of the
// transform at position dft_slot(k, log2L)).  Both take two radix-2 stages per pass, as one
// radix-4 butterfly (three twiddle products per four values).
template <typename T>
__device__ __forceinline__ void fft_lines(Cplx<T>* s, Cplx<T>* tmp, int count, int L, int log2L, const Cplx<T>* tw,
                                          bool inverse, bool dif) {
  const int tid = threadIdx.x, nth = blockDim.x;
  if (log2L < 0) {
    for (int i = tid; i < count * L; i += nth) {
      const int c = i / L, k = i - c * L;
      const Cplx<T>* x = s + c * L;
      T re = T(0), im = T(0);
      int m = 0;  // (j * k) mod L
      for (int j = 0; j < L; ++j) {
        Cplx<T> w = tw[m];
        if (inverse) w.im = -w.im;
        const Cplx<T> v = cmul(w, x[j]);
        re += v.re;
        im += v.im;
        m += k;
        if (m >= L) m -= L;
      }
      tmp[i] = Cplx<T>{re, im};
    }
    __syncthreads();
    for (int i = tid; i < count * L; i += nth) s[i] = tmp[i];
    __syncthreads();
    return;
  }
  if (log2L == 0) return;
  const int q = L >> 2;  // radix-2^2 butterflies per line and pass
  if (!dif) {
    int half = 1, lh = 0;
    if (log2L & 1) {  // one radix-2 stage (span 1) first
      const int hl = L >> 1;
      for (int t = tid; t < count * hl; t += nth) {
        Cplx<T>* b = s + (t >> (log2L - 1)) * L + 2 * (t & (hl - 1));
        const Cplx<T> u = b[0], v = b[1];
        b[0] = cadd(u, v);
        b[1] = csub(u, v);
      }
      __syncthreads();
      half = 2;
      lh = 1;
    }
    if (half == 1 && L >= 4) {  // the first pass: every twiddle is 1
      for (int t = tid; t < count * q; t += nth) {
        Cplx<T>* b = s + (t >> (log2L - 2)) * L + 4 * (t & (q - 1));
        const Cplx<T> a = b[0], bb = b[1], c = b[2], d = b[3];
        const Cplx<T> A1 = cadd(a, bb), B1 = csub(a, bb), C1 = cadd(c, d);
        Cplx<T> D1 = csub(c, d);
        D1 = inverse ? Cplx<T>{-D1.im, D1.re} : Cplx<T>{D1.im, -D1.re};
        b[0] = cadd(A1, C1);
        b[2] = csub(A1, C1);
        b[1] = cadd(B1, D1);
        b[3] = csub(B1, D1);
      }
      __syncthreads();
      half = 4;
      lh = 2;
    }
    // two stages (spans half, 2 half) as one radix-4 butterfly with the three twiddles
    // W^p, W^2p, W^3p (W = exp(-+ 2 pi i / 4 half), p the position in the group)
    for (; half < L; half <<= 2, lh += 2) {
      const int s4 = L / (4 * half);
      for (int t = tid; t < count * q; t += nth) {
        const int line = t >> (log2L - 2), tt = t & (q - 1);
        const int grp = tt >> lh, pos = tt & (half - 1);
        Cplx<T>* b = s + line * L + grp * 4 * half + pos;
        Cplx<T> w1 = tw[pos * s4], w2 = tw[2 * pos * s4], w3 = tw[3 * pos * s4];
        if (inverse) {
          w1.im = -w1.im;
          w2.im = -w2.im;
          w3.im = -w3.im;
        }
        const Cplx<T> a = b[0], tb = cmul(w2, b[half]);
        const Cplx<T> tc = cmul(w1, b[2 * half]), td = cmul(w3, b[3 * half]);
        const Cplx<T> s1 = cadd(a, tb), s2 = csub(a, tb), s3 = cadd(tc, td);
        Cplx<T> s4v = csub(tc, td);
        s4v = inverse ? Cplx<T>{-s4v.im, s4v.re} : Cplx<T>{s4v.im, -s4v.re};  // times -+ i
        b[0] = cadd(s1, s3);
        b[2 * half] = csub(s1, s3);
        b[half] = cadd(s2, s4v);
        b[3 * half] = csub(s2, s4v);
      }
      __syncthreads();
    }
  } else {
    // spans 2h and h per pass, from 2h = L / 2 down; a last span-1 stage if log2L is odd
    int h = q, lh = log2L - 2, stages = log2L;
    for (; stages >= 2; h >>= 2, lh -= 2, stages -= 2) {
      if (h == 1) {  // the last pass: every twiddle is 1
        for (int t = tid; t < count * q; t += nth) {
          Cplx<T>* b = s + (t >> (log2L - 2)) * L + 4 * (t & (q - 1));
          const Cplx<T> x0 = b[0], x1 = b[1], x2 = b[2], x3 = b[3];
          const Cplx<T> y0 = cadd(x0, x2), y1 = cadd(x1, x3), y2 = csub(x0, x2);
          Cplx<T> y3 = csub(x1, x3);
          y3 = inverse ? Cplx<T>{-y3.im, y3.re} : Cplx<T>{y3.im, -y3.re};
          b[0] = cadd(y0, y1);
          b[1] = csub(y0, y1);
          b[2] = cadd(y2, y3);
          b[3] = csub(y2, y3);
        }
        __syncthreads();
        continue;
      }
      // the two stages as one radix-4 butterfly with the three twiddles W^p, W^2p, W^3p
      const int s4 = L / (4 * h);
      for (int t = tid; t < count * q; t += nth) {
        const int line = t >> (log2L - 2), tt = t & (q - 1);
        const int grp = tt >> lh, pos = tt & (h - 1);
        Cplx<T>* b = s + line * L + grp * 4 * h + pos;
        Cplx<T> w1 = tw[pos * s4], w2 = tw[2 * pos * s4], w3 = tw[3 * pos * s4];
        if (inverse) {
          w1.im = -w1.im;
          w2.im = -w2.im;
          w3.im = -w3.im;
        }
        const Cplx<T> x0 = b[0], x1 = b[h], x2 = b[2 * h], x3 = b[3 * h];
        const Cplx<T> u0 = cadd(x0, x2), u1 = cadd(x1, x3), u2 = csub(x0, x2);
        Cplx<T> u3 = csub(x1, x3);
        u3 = inverse ? Cplx<T>{-u3.im, u3.re} : Cplx<T>{u3.im, -u3.re};  // times -+ i
        b[0] = cadd(u0, u1);
        b[h] = cmul(w2, csub(u0, u1));
        b[2 * h] = cmul(w1, cadd(u2, u3));
        b[3 * h] = cmul(w3, csub(u2, u3));
      }
      __syncthreads();
    }
    if (stages == 1) {
      const int hl = L >> 1;
      for (int t = tid; t < count * hl; t += nth) {
        Cplx<T>* b = s + (t >> (log2L - 1)) * L + 2 * (t & (hl - 1));
        const Cplx<T> u = b[0], v = b[1];
        b[0] = cadd(u, v);
        b[1] = csub(u, v);
      }
      __syncthreads();
    }
  }
}

}  // namespace dgk
