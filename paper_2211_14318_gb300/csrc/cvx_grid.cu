// cvx_grid.cu -- the global-grid form of the method (Secs. 4.1-4.3, 5.1-5.3,
// 6.1, 6.8): Eq. (4.3) iterated on the cuboid deformation-gradient grid of
// Sec. 5.2 for F in R^{2x2} or R^{3x3} (four or nine components) with a set
// of grid-index directions (the reduced set R^1_1 of Eq. 5.1), the
// one-dimensional convexification of Algorithm 1 on every rank-one line of
// the grid, the lamination forest, and Algorithm 2's trees (with the
// multilinear-interpolation branching of Sec. 5.3) evaluated by Algorithm 3
// at arbitrary points.  Energies: Eq. (2.9) over Eq. (2.3) (Neo-Hooke) or
// Eq. (2.2) (St. Venant-Kirchhoff), and the double-well test energy.
//
// Design.  For a direction R every grid point lies on exactly one maximal
// line {F + l R} of the grid, and all points of one line share the line's
// lower hull: the value of Eq. (4.3) at a point is the hull read at that
// point.  So one thread builds Algorithm 1's hull of one (direction, line)
// pair once (a stack in shared memory) and then walks the line again: a
// point strictly inside a hull edge records the numerator of its chord value
// and the edge's ends.  The per-point minimum over the directions (lowest
// direction index on equal values, a strict decrease required) is a second
// kernel over the points; it divides only where a direction can still win
// (a product with the rounded reciprocal of the integer denominator bounds
// the quotient from below first).  Predicates and chord values are the FP64
// expressions of the hull at the point with every operation rounded on its
// own (no contraction into FMA): the hull's vertex set does not depend on
// where the line is read, so each step is reproducible bit for bit.
// The global iteration stops on the device: a one-thread kernel after each
// step sets a flag once the largest decrease is at most tol, and the kernels
// of the later steps return at once, so the host enqueues kmax steps without
// waiting on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "cvx_handle.h"

namespace cvx {
namespace {

constexpr int kGridMaxDirs = 4096;   // directions per call
constexpr int kGridMaxIters = 64;    // global iterations (lamination orders) per call
constexpr int kGridMaxLine = 512;    // grid points per component (longest line)
constexpr size_t kGridChunkBytes = (size_t)1 << 30;  // per-direction line results per chunk

// Bytes of line results per chunk of directions: kGridChunkBytes, or the
// environment variable CVX_GRID_CHUNK_BYTES (smaller chunks, for tests).
size_t grid_chunk_bytes() {
    const char *e = getenv("CVX_GRID_CHUNK_BYTES");
    if (e && *e) {
        const long long v = atoll(e);
        if (v > 0) return (size_t)v;
    }
    return kGridChunkBytes;
}

template <int D>
struct GridT {
    int n[D];
    int s[D];  // flat-index strides (last component fastest)
    double lo[D], delta[D];
    int N;
};

template <int D>
struct GridDirT {
    int o[D];  // grid-index offset of one step along the line
    int step;  // its flat-index step
};

__device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Key of a non-NaN double whose signed-integer order is the order of the
// values (-0 and +0 share the key 0): the comparisons of the hull run on the
// integer pipe and leave the FP64 pipe to the arithmetic.
__device__ __forceinline__ long long order_key(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

// Exact double of a nonzero integer with |v| < 2^20, assembled on the integer
// pipe from the IEEE-754 binary64 layout (sign, biased exponent, fraction).
__device__ __forceinline__ double exact_double(int v) {
    const unsigned a = (unsigned)(v < 0 ? -v : v);
    const int e = 31 - __clz(a);  // a in [2^e, 2^(e+1))
    const unsigned long long frac = ((unsigned long long)a << (52 - e)) & ((1ull << 52) - 1);
    unsigned long long bits = ((unsigned long long)(1023 + e) << 52) | frac;
    if (v < 0) bits |= 1ull << 63;
    return __longlong_as_double((long long)bits);
}

template <int D>
__device__ __forceinline__ void grid_index(const GridT<D> &g, int idx, int *i) {
#pragma unroll
    for (int c = D - 1; c >= 0; --c) {
        i[c] = idx % g.n[c];
        idx /= g.n[c];
    }
}

// Grid point F_c = lo_c + i_c delta_c, each operation rounded on its own.
template <int D>
__device__ __forceinline__ void grid_point(const GridT<D> &g, int idx, double *F) {
    int i[D];
    grid_index<D>(g, idx, i);
#pragma unroll
    for (int c = 0; c < D; ++c) F[c] = __dadd_rn(g.lo[c], __dmul_rn((double)i[c], g.delta[c]));
}

// Eq. (2.9) in s = psi0: s <= beta: (1 - D(beta)) (s - beta); otherwise
// (1 - D_inf)(s - beta) + D_inf D_0 (e^{-beta/D_0} - e^{-s/D_0}).
__device__ __forceinline__ double w_of_psi0(double s, double beta, const Material &m) {
    const double ek = exp(-beta / m.D0);
    if (s <= beta) return (1.0 - m.Dinf * (1.0 - ek)) * (s - beta);
    return (1.0 - m.Dinf) * (s - beta) + m.Dinf * m.D0 * (ek - exp(-s / m.D0));
}

// Invariants of C = F^T F (Sec. 2) for F in R^{dxd}, D = d^2, row-major:
// I1 = tr C, I2 = the sum of the principal 2x2 minors of C, J = det F; d = 2
// is plane strain (C33 = 1: I1 gains 1, I2 gains C11 + C22).
template <int D>
__device__ void invariants(const double *F, double &I1, double &I2, double &J, double *C) {
    if (D == 4) {
        C[0] = F[0] * F[0] + F[2] * F[2];
        C[1] = F[0] * F[1] + F[2] * F[3];
        C[2] = C[1];
        C[3] = F[1] * F[1] + F[3] * F[3];
        I1 = C[0] + C[3] + 1.0;
        I2 = (C[0] * C[3] - C[1] * C[1]) + C[0] + C[3];
        J = __dsub_rn(__dmul_rn(F[0], F[3]), __dmul_rn(F[1], F[2]));
    } else {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                C[3 * a + b] = F[a] * F[b] + F[3 + a] * F[3 + b] + F[6 + a] * F[6 + b];
        I1 = C[0] + C[4] + C[8];
        I2 = (C[0] * C[4] - C[1] * C[3]) + (C[0] * C[8] - C[2] * C[6]) +
             (C[4] * C[8] - C[5] * C[7]);
        // each operation rounded on its own, in the oracle's order: which
        // points count as det F <= 0 must not depend on FMA contraction
        const double m0 = __dsub_rn(__dmul_rn(F[4], F[8]), __dmul_rn(F[5], F[7]));
        const double m1 = __dsub_rn(__dmul_rn(F[3], F[8]), __dmul_rn(F[5], F[6]));
        const double m2 = __dsub_rn(__dmul_rn(F[3], F[7]), __dmul_rn(F[4], F[6]));
        J = __dadd_rn(__dsub_rn(__dmul_rn(F[0], m0), __dmul_rn(F[1], m1)), __dmul_rn(F[2], m2));
    }
}

// psi0 (Eq. 2.3 with ln|J|, or Eq. 2.2) and whether det F <= 0 excludes F
// under the rule: 0 excludes det F <= 0; 1 keeps det F < 0 for Eq. (2.3)
// (ln|det F|) and every F for Eq. (2.2) (a polynomial).
template <int D>
__device__ bool psi0_grid(const double *F, const Material &m, int rule, double &s, double &J,
                          double &I1, double *C) {
    double I2;
    invariants<D>(F, I1, I2, J, C);
    if (m.energy == CVX_ENERGY_STVK_DAMAGE) {
        s = m.lam / 8.0 * (I1 - 3.0) * (I1 - 3.0) + m.mu / 4.0 * (I1 * I1 - 2.0 * I1 - 2.0 * I2 + 3.0);
        return rule == 0 && !(J > 0.0);
    }
    const double aj = fabs(J);
    const double lj = log(aj);
    s = 0.5 * m.mu * (I1 - 3.0) - m.mu * lj + 0.5 * m.lam * lj * lj;
    return rule == 0 ? !(J > 0.0) : !(aj > 0.0);
}

template <int D>
__device__ double grid_w64(const double *F, double beta, const Material &m, int rule) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) return D == 4 ? energy64(F, beta, m) : nan("");
    double s, J, I1, C[D];
    if (psi0_grid<D>(F, m, rule, s, J, I1, C)) return nan("");
    return w_of_psi0(s, beta, m);
}

// dW/dF = (1 - D(max(s, beta))) dpsi0/dF with
//   Eq. (2.3): mu F - mu F^-T + lambda ln|J| F^-T (d ln|J|/dF = F^-T = cof F / J);
//   Eq. (2.2): F (lambda/2 (I1 - 3) 1 + mu (C - 1)).
template <int D>
__device__ void grid_p64(const double *F, double beta, const Material &m, int rule, double *P) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        if (D == 4) stress64(F, beta, m, P);
        else
            for (int c = 0; c < D; ++c) P[c] = nan("");
        return;
    }
    double s, J, I1, C[D];
    if (psi0_grid<D>(F, m, rule, s, J, I1, C)) {
        for (int c = 0; c < D; ++c) P[c] = nan("");
        return;
    }
    const double b = s > beta ? s : beta;
    const double gd = 1.0 - m.Dinf * (1.0 - exp(-b / m.D0));
    constexpr int d = D == 4 ? 2 : 3;
    if (m.energy == CVX_ENERGY_STVK_DAMAGE) {
        double S[D];
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c)
                S[d * a + c] = m.mu * (C[d * a + c] - (a == c ? 1.0 : 0.0)) +
                               (a == c ? 0.5 * m.lam * (I1 - 3.0) : 0.0);
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c) {
                double v = 0.0;
                for (int k = 0; k < d; ++k) v += F[d * a + k] * S[d * k + c];
                P[d * a + c] = gd * v;
            }
        return;
    }
    double cof[D];
    if (D == 4) {
        cof[0] = F[3];
        cof[1] = -F[2];
        cof[2] = -F[1];
        cof[3] = F[0];
    } else {
        cof[0] = F[4] * F[8] - F[5] * F[7];
        cof[1] = F[5] * F[6] - F[3] * F[8];
        cof[2] = F[3] * F[7] - F[4] * F[6];
        cof[3] = F[2] * F[7] - F[1] * F[8];
        cof[4] = F[0] * F[8] - F[2] * F[6];
        cof[5] = F[1] * F[6] - F[0] * F[7];
        cof[6] = F[1] * F[5] - F[2] * F[4];
        cof[7] = F[2] * F[3] - F[0] * F[5];
        cof[8] = F[0] * F[4] - F[1] * F[3];
    }
    const double lj = log(fabs(J));
    for (int c = 0; c < D; ++c) {
        const double fit = cof[c] / J;
        P[c] = gd * (m.mu * F[c] - m.mu * fit + m.lam * lj * fit);
    }
}

// d^2W/dFdF (D x D, A[D a + b] = dP_a / dF_b over the row-major entries):
// A = g d^2psi0 + g' dpsi0 (x) dpsi0, g = 1 - D(max(s, beta)), on loading
// (s > beta) g' = -(D_inf / D_0) e^{-s / D_0}, with
//   Eq. (2.3), G = F^-T, ln|J|:
//     d^2psi0/dF_iJ dF_kL = mu d_ik d_JL + lambda G_iJ G_kL + (mu - lambda ln|J|) G_iL G_kJ;
//   Eq. (2.2), S = lambda/2 (I1 - 3) 1 + mu (C - 1), dpsi0/dF = F S:
//     d^2psi0/dF_iJ dF_kL = d_ik S_LJ + lambda F_iJ F_kL + mu F_iL F_kJ + mu (F F^T)_ik d_JL.
template <int D>
__device__ void grid_a64(const double *F, double beta, const Material &m, int rule, double *A) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        if (D == 4) tangent64(F, beta, m, A);
        else
            for (int c = 0; c < D * D; ++c) A[c] = nan("");
        return;
    }
    double s, J, I1, C[D];
    if (psi0_grid<D>(F, m, rule, s, J, I1, C)) {
        for (int c = 0; c < D * D; ++c) A[c] = nan("");
        return;
    }
    constexpr int d = D == 4 ? 2 : 3;
    const double b = s > beta ? s : beta;
    const double g = 1.0 - m.Dinf * (1.0 - exp(-b / m.D0));
    const double gp = s > beta ? -(m.Dinf / m.D0) * exp(-s / m.D0) : 0.0;
    double dp[D];
    grid_p64<D>(F, beta, m, rule, dp);  // g dpsi0/dF
    const double ig = 1.0 / g;
    for (int c = 0; c < D; ++c) dp[c] *= ig;
    if (m.energy == CVX_ENERGY_STVK_DAMAGE) {
        double S[D], FF[D];
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c) {
                double v = 0.0;
                for (int k = 0; k < d; ++k) v += F[d * a + k] * F[d * c + k];
                FF[d * a + c] = v;
                S[d * a + c] = m.mu * (C[d * a + c] - (a == c ? 1.0 : 0.0)) +
                               (a == c ? 0.5 * m.lam * (I1 - 3.0) : 0.0);
            }
        for (int i = 0; i < d; ++i)
            for (int jj = 0; jj < d; ++jj)
                for (int k = 0; k < d; ++k)
                    for (int l = 0; l < d; ++l) {
                        const double d2 = (i == k ? S[d * l + jj] : 0.0) +
                                          m.lam * F[d * i + jj] * F[d * k + l] +
                                          m.mu * F[d * i + l] * F[d * k + jj] +
                                          (jj == l ? m.mu * FF[d * i + k] : 0.0);
                        A[D * (d * i + jj) + d * k + l] =
                            g * d2 + gp * dp[d * i + jj] * dp[d * k + l];
                    }
        return;
    }
    double G[D];
    if (D == 4) {
        G[0] = F[3] / J;
        G[1] = -F[2] / J;
        G[2] = -F[1] / J;
        G[3] = F[0] / J;
    } else {
        G[0] = (F[4] * F[8] - F[5] * F[7]) / J;
        G[1] = (F[5] * F[6] - F[3] * F[8]) / J;
        G[2] = (F[3] * F[7] - F[4] * F[6]) / J;
        G[3] = (F[2] * F[7] - F[1] * F[8]) / J;
        G[4] = (F[0] * F[8] - F[2] * F[6]) / J;
        G[5] = (F[1] * F[6] - F[0] * F[7]) / J;
        G[6] = (F[1] * F[5] - F[2] * F[4]) / J;
        G[7] = (F[2] * F[3] - F[0] * F[5]) / J;
        G[8] = (F[0] * F[4] - F[1] * F[3]) / J;
    }
    const double cc = m.mu - m.lam * log(fabs(J));
    for (int i = 0; i < d; ++i)
        for (int jj = 0; jj < d; ++jj)
            for (int k = 0; k < d; ++k)
                for (int l = 0; l < d; ++l) {
                    const double d2 = (i == k && jj == l ? m.mu : 0.0) +
                                      m.lam * G[d * i + jj] * G[d * k + l] +
                                      cc * G[d * i + l] * G[d * k + jj];
                    A[D * (d * i + jj) + d * k + l] = g * d2 + gp * dp[d * i + jj] * dp[d * k + l];
                }
}

// Number of grid points on the line that starts at index i along offset o.
template <int D>
__device__ __forceinline__ int line_length(const GridT<D> &g, const int *i, const int *o) {
    int len = 1 << 30;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        if (o[c] > 0) len = min(len, (g.n[c] - 1 - i[c]) / o[c]);
        else if (o[c] < 0) len = min(len, i[c] / (-o[c]));
    }
    return len + 1;
}

// W^0 on the grid.
template <int D>
__global__ void k_grid_energy(GridT<D> g, Material m, double beta, int rule, double *W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    double F[D];
    grid_point<D>(g, p, F);
    W[p] = grid_w64<D>(F, beta, m, rule);
}

// Line starts: per point (one index decomposition) and direction j, the point
// starts a line if its predecessor along j lies outside the grid.  The starts
// of region j of `starts` (line_off[j] .. line_off[j + 1]) are ordered by
// line length, longest first, so that a warp of the line kernel takes lines
// of one length (a counting sort: phase 0 counts the lines of each
// (direction, length) in hist, k_grid_len_scan turns the counts into
// offsets, phase 1 places each start at its offset; the order among lines of
// one length is arbitrary and changes no result).  Lanes of a warp with the
// same (direction, length) share one atomic.  The direction offsets are
// staged in shared memory.
template <int D>
__global__ void k_grid_starts(GridT<D> g, const GridDirT<D> *dirs, int nd,
                              const long long *line_off, unsigned *hist, int cap, int phase,
                              int *starts) {
    extern __shared__ int soff[];  // nd x D offsets
    for (int k = threadIdx.x; k < nd * D; k += blockDim.x) soff[k] = dirs[k / D].o[k % D];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < g.N;
         b += (long long)gridDim.x * blockDim.x) {
        const long long p = b + threadIdx.x;
        const bool valid = p < g.N;
        int i[D];
        if (valid) grid_index<D>(g, (int)p, i);
        for (int j = 0; j < nd; ++j) {
            bool st = false;
            int len = 0;
            if (valid) {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const int q = i[c] - soff[j * D + c];
                    st |= (q < 0) || (q >= g.n[c]);
                }
                if (st) len = line_length<D>(g, i, soff + j * D);
            }
            const unsigned act = __ballot_sync(0xffffffffu, st);
            if (!st) continue;
            const unsigned grp = __match_any_sync(act, len);
            const int leader = __ffs(grp) - 1;
            unsigned* cell = hist + (size_t)j * (cap + 1) + len;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(cell, (unsigned)__popc(grp));
            base = __shfl_sync(grp, base, leader);
            if (phase == 1)
                starts[line_off[j] + base + __popc(grp & ((1u << lane) - 1))] = (int)p;
        }
    }
}

// Per direction: the counts of lines of each length become the offsets of
// their first line in the region, longest lines first.
__global__ void k_grid_len_scan(int nd, int cap, unsigned *hist) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nd) return;
    unsigned *h = hist + (size_t)j * (cap + 1);
    unsigned acc = 0;
    for (int len = cap; len >= 0; --len) {
        const unsigned c = h[len];
        h[len] = acc;
        acc += c;
    }
}

// One thread per (direction, line) of directions [j0, j1): Algorithm 1 on the
// finite values of W_in along the line (stack in shared memory, layout
// [slot][thread]), then every point of the line reads the hull there:
//   a hull vertex keeps its own value (no split, S = 0);
//   a point strictly between vertices a < x < b, with x_a, x_b taken relative
//   to the point (x_a < 0 < x_b), records the numerator x_b w_a - x_a w_b of
//   its chord value h = (x_b w_a - x_a w_b) / (x_b - x_a) in H and the pair
//   (x_a, x_b) as two 16-bit fields in S.
// Non-finite points keep their value.  H and S are chunk-major: entry
// (j - j0) N + point.
template <int D>
__global__ void __launch_bounds__(128) k_grid_lines(GridT<D> g, const GridDirT<D> *dirs,
                                                    const long long *line_off, int j0, int j1,
                                                    const int *starts, const double *Win,
                                                    double *H, unsigned *S, int cap,
                                                    const int *done) {
    if (done && *done) return;
    extern __shared__ double gsm[];
    const int T = blockDim.x;
    const long long t = line_off[j0] + (long long)blockIdx.x * T + threadIdx.x;
    if (t >= line_off[j1]) return;
    int lo = j0, hi = j1 - 1;  // the region holding t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (line_off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int j = lo;
    const GridDirT<D> d = dirs[j];
    const int p0 = starts[t];
    int i0[D];
    grid_index<D>(g, p0, i0);
    const int len = line_length<D>(g, i0, d.o);
    double *sv = gsm + threadIdx.x;
    short *sx = reinterpret_cast<short *>(gsm + (size_t)cap * T) + threadIdx.x;

    // Algorithm 1: monotone chain over the finite values, pops while the top
    // of the stack is not strictly below the chord to the new point
    int k = 0;
    for (int l = 0; l < len; ++l) {
        const double w = Win[p0 + l * d.step];
        if (!finite_bits(w)) continue;
        while (k >= 2) {
            const double wp = sv[(k - 2) * T], wq = sv[(k - 1) * T];
            const int xp = sx[(k - 2) * T], xq = sx[(k - 1) * T];
            const double A = __dsub_rn(wq, wp), B = __dsub_rn(w, wq);
            const int di = l - xq, dp = xq - xp;
            // multiplying by 1 is exact: skip it
            const double lhs = di == 1 ? A : __dmul_rn(A, exact_double(di));
            const double rhs = dp == 1 ? B : __dmul_rn(B, exact_double(dp));
            if (order_key(lhs) >= order_key(rhs)) --k;
            else break;
        }
        sv[k * T] = w;
        sx[k * T] = (short)l;
        ++k;
    }
    // every finite point lies between the first and the last vertex
    const long long base = (long long)(j - j0) * g.N;
    int e = 0;
    for (int l = 0; l < len; ++l) {
        const int idx = p0 + l * d.step;
        double num = 0.0;
        unsigned sp = 0;
        if (k > 1) {
            while (e + 2 < k && sx[(e + 1) * T] <= l) ++e;
            const int xa = sx[e * T], xb = sx[(e + 1) * T];
            // strictly inside the edge (and finite: a non-finite point is no
            // vertex, but a hole can lie inside an edge)
            if (xa < l && l < xb && finite_bits(Win[idx])) {
                const int ra = xa - l, rb = xb - l;
                num = __dsub_rn(__dmul_rn(exact_double(rb), sv[e * T]),
                                __dmul_rn(exact_double(ra), sv[(e + 1) * T]));
                sp = ((unsigned)ra & 0xffffu) | ((unsigned)rb << 16);
            }
        }
        H[base + idx] = num;
        S[base + idx] = sp;
    }
}

// rcp[v] = fl(1 / v), v = 1 .. 2 kGridMaxLine (the chord denominators).
__global__ void k_grid_rcp(double *rcp) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v <= 2 * kGridMaxLine) rcp[v] = v ? __drcp_rn((double)v) : 0.0;
}

// Per point, directions [j0, j1) in order: the first strict decrease below
// the best so far wins (first chunk: the best so far is W_in itself, no
// split).  The chord value h = fl(num / den) is needed only where it can win:
// q = fl(num fl(1/den)) is within 3.4e-16 |q| of h, so fl(q (1 -+ 5e-16)) is
// a lower bound of h and a direction whose bound is not below the best so far
// cannot win; the others are divided exactly and compared.  lam = (dir, l-,
// l+) per point (dir = -1: no split).  The last chunk adds the point's
// decrease W_in - W_out to the step's maximum (dec, as the bits of a
// non-negative double).
__global__ void k_grid_reduce(int N, int j0, int j1, int first, int last, const double *Win,
                              const double *H, const unsigned *S, const double *rcp,
                              double *Wout, int *lam, unsigned long long *dec, const int *done) {
    if (done && *done) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long dbits = 0;
    if (p < N) {
        const double w0 = Win[p];
        double best = w0;
        int bd = -1, bm = 0, bp = 0;
        if (!first) {
            best = Wout[p];
            bd = lam[3 * p];
            bm = lam[3 * p + 1];
            bp = lam[3 * p + 2];
        }
        for (int j = j0; j < j1; ++j) {
            const long long e = (long long)(j - j0) * N + p;
            const unsigned s = S[e];
            if (s) {
                const double num = H[e];
                const int ra = (int)(short)(s & 0xffffu), rb = (int)(s >> 16);
                const double q = __dmul_rn(num, rcp[rb - ra]);
                const double lb =
                    __dmul_rn(q, __double_as_longlong(q) < 0 ? 1.0 + 5e-16 : 1.0 - 5e-16);
                if (order_key(lb) < order_key(best)) {
                    const double h = __ddiv_rn(num, exact_double(rb - ra));
                    if (order_key(h) < order_key(best)) {
                        best = h;
                        bd = j;
                        bm = ra;
                        bp = rb;
                    }
                }
            }
        }
        Wout[p] = best;
        lam[3 * p] = bd;
        lam[3 * p + 1] = bm;
        lam[3 * p + 2] = bp;
        if (last && finite_bits(w0) && finite_bits(best))
            dbits = (unsigned long long)__double_as_longlong(__dsub_rn(w0, best));
    }
    if (!last || !dec) return;
    // non-negative doubles order like their bit patterns: reduce on the integer pipe
    for (int o = 16; o; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, dbits, o);
        dbits = v > dbits ? v : dbits;
    }
    if ((threadIdx.x & 31) == 0 && dbits) atomicMax(dec, dbits);
}

// After step k: the step count so far, and the stop flag once the step's
// largest decrease is at most tol (Sec. 4.1's stopping rule).
__global__ void k_grid_check(const unsigned long long *dec_k, double tol, int *done, int *iters,
                             int k) {
    if (*done) return;
    *iters = k + 1;
    if (__longlong_as_double((long long)*dec_k) <= tol) *done = 1;
}

// W^K ends in the ping buffer when K is odd: copy it to the output.
__global__ void k_grid_final(int N, const int *iters, const double *pong, double *W) {
    if ((*iters & 1) == 0) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) W[p] = pong[p];
}

// Trees of Algorithm 2 tabulated per grid point and order (Algorithm 3 by
// dynamic programming over the orders).  T_d(p) = (W, P, leaves) of the tree
// below grid point p at order d: at d = 0 (or where no iteration up to d
// split p) the leaf values W(p), P(p) (Eq. 2.12) and one leaf; where
// iteration d split p with record (dir, l-, l+), xi = -l- / (l+ - l-),
//   T_d(p) = (1 - xi) T_{d-1}(p + l- R) + xi T_{d-1}(p + l+ R);
// elsewhere T_d(p) = T_{d-1}(p) (the latest split below d decides).  A record
// this library did not write makes p a leaf at that order.  Layout: W[N],
// P[D][N], leaves[N] per order, ping-pong between two buffers.
template <int D>
__global__ void k_grid_tree0(GridT<D> g, Material m, double beta, int rule, double *Tw,
                             double *Tp, long long *Tl, double *Ta) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    double F[D], P[D];
    grid_point<D>(g, p, F);
    Tw[p] = grid_w64<D>(F, beta, m, rule);
    grid_p64<D>(F, beta, m, rule, P);
    for (int c = 0; c < D; ++c) Tp[(long long)c * g.N + p] = P[c];
    Tl[p] = 1;
    if (Ta) {
        double A[D * D];
        grid_a64<D>(F, beta, m, rule, A);
        for (int c = 0; c < D * D; ++c) Ta[(long long)c * g.N + p] = A[c];
    }
}

template <int D>
__global__ void k_grid_tree_step(GridT<D> g, const GridDirT<D> *dirs, int nd, const int *rec,
                                 const double *Tw0, const double *Tp0, const long long *Tl0,
                                 const double *Tw, const double *Tp, const long long *Tl,
                                 double *Uw, double *Up, long long *Ul, const double *Ta0,
                                 const double *Ta, double *Ua) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    const long long N = g.N;
    const int dj = rec[3 * (long long)p], lm = rec[3 * (long long)p + 1],
              lp = rec[3 * (long long)p + 2];
    if (dj < 0) {  // not split in this iteration: the tree of the order below
        Uw[p] = Tw[p];
        for (int c = 0; c < D; ++c) Up[c * N + p] = Tp[c * N + p];
        Ul[p] = Tl[p];
        if (Ua)
            for (int c = 0; c < D * D; ++c) Ua[c * N + p] = Ta[c * N + p];
        return;
    }
    const int step = dj < nd ? dirs[dj].step : 0;
    const long long cm = p + (long long)lm * step, cp = p + (long long)lp * step;
    if (dj >= nd || !(lm < 0 && lp > 0) || cm < 0 || cm >= N || cp < 0 || cp >= N) {
        Uw[p] = Tw0[p];
        for (int c = 0; c < D; ++c) Up[c * N + p] = Tp0[c * N + p];
        Ul[p] = Tl0[p];
        if (Ua)
            for (int c = 0; c < D * D; ++c) Ua[c * N + p] = Ta0[c * N + p];
        return;
    }
    const double xi = __ddiv_rn((double)(-lm), (double)(lp - lm));
    const double xm = __dsub_rn(1.0, xi);
    Uw[p] = __dadd_rn(__dmul_rn(xm, Tw[cm]), __dmul_rn(xi, Tw[cp]));
    for (int c = 0; c < D; ++c)
        Up[c * N + p] = __dadd_rn(__dmul_rn(xm, Tp[c * N + cm]), __dmul_rn(xi, Tp[c * N + cp]));
    if (Ua)
        for (int c = 0; c < D * D; ++c)
            Ua[c * N + p] =
                __dadd_rn(__dmul_rn(xm, Ta[c * N + cm]), __dmul_rn(xi, Ta[c * N + cp]));
    const long long l = Tl[cm] + Tl[cp];
    Ul[p] = l < Tl[cm] ? 0x7fffffffffffffffLL : l;  // saturates
}

// Algorithm 2's tree at n points evaluated by Algorithm 3, one thread per
// point: the corners of the grid cell holding F (multilinear weights
// prod_c (1 - t_c or t_c); a coordinate within 1e-12 grid steps of a grid
// value counts as on it; corners of weight 0 left out; corner bit c counted
// from the first component) at order K, each contributing its weight times
// the tabulated tree T_K.  W_interp is the multilinear interpolation of W^K.
template <int D>
__global__ void k_grid_query(GridT<D> g, const double *WK, const double *Tw, const double *Tp,
                             const long long *Tl, const double *Ta, long long n,
                             const double *F, double *Wi, double *Wt, double *P, double *A,
                             long long *leaves) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int i0[D];
    double t[D];
    bool inside = true;
    for (int c = 0; c < D; ++c) {
        const double u = __ddiv_rn(__dsub_rn(F[D * q + c], g.lo[c]), g.delta[c]);
        if (u < -1e-12 || u > (double)(g.n[c] - 1) + 1e-12) inside = false;
        double f = floor(u);
        double r = __dsub_rn(u, f);
        if (r > 1.0 - 1e-12) {
            f = __dadd_rn(f, 1.0);
            r = 0.0;
        } else if (r < 1e-12) {
            r = 0.0;
        }
        int ii = (int)f;
        ii = ii > g.n[c] - 1 ? g.n[c] - 1 : ii;
        ii = ii < 0 ? 0 : ii;
        i0[c] = ii;
        t[c] = r;
    }
    double wi = 0.0, wt = 0.0, Pp[D];
    for (int c = 0; c < D; ++c) Pp[c] = 0.0;
    if (A)
        for (int c = 0; c < D * D; ++c) A[(long long)D * D * q + c] = 0.0;
    long long nl = 0;
    const long long N = g.N;
    for (int corner = 0; inside && corner < (1 << D); ++corner) {
        double w = 1.0;
        int flat = 0;
        for (int c = 0; c < D; ++c) {
            const int up = (corner >> (D - 1 - c)) & 1;
            w = __dmul_rn(w, up ? t[c] : __dsub_rn(1.0, t[c]));
            flat += (i0[c] + up) * g.s[c];
        }
        if (w == 0.0) continue;
        wi = __dadd_rn(wi, __dmul_rn(w, WK[flat]));
        wt = __dadd_rn(wt, __dmul_rn(w, Tw[flat]));
        for (int a = 0; a < D; ++a) Pp[a] = __dadd_rn(Pp[a], __dmul_rn(w, Tp[a * N + flat]));
        nl += Tl[flat];
        if (A)  // accumulated in place (the output row starts at zero)
            for (int c = 0; c < D * D; ++c)
                A[(long long)D * D * q + c] =
                    __dadd_rn(A[(long long)D * D * q + c], __dmul_rn(w, Ta[c * N + flat]));
    }
    if (!inside) {
        wi = wt = nan("");
        for (int a = 0; a < D; ++a) Pp[a] = nan("");
        if (A)
            for (int c = 0; c < D * D; ++c) A[(long long)D * D * q + c] = nan("");
    }
    Wi[q] = wi;
    Wt[q] = wt;
    for (int a = 0; a < D; ++a) P[D * q + a] = Pp[a];
    if (leaves) leaves[q] = nl;
}

// ------------------------------------------------------------------ host

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int D>
int check_grid(const cvx_grid *g, GridT<D> &gd) {
    long long N = 1;
    for (int c = 0; c < D; ++c) {
        if (g->n[c] < 1 || g->n[c] > kGridMaxLine)
            return fail(CVX_ERR_INVALID_ARG, "grid points per component must be in [1, %d]",
                        kGridMaxLine);
        if (!(g->delta[c] > 0.0) || !isfinite(g->delta[c]) || !isfinite(g->lo[c]))
            return fail(CVX_ERR_INVALID_ARG, "grid spacing must be positive and bounds finite");
        N *= g->n[c];
        if (N > 0x7fffffffLL)
            return fail(CVX_ERR_INVALID_ARG, "grid has more than 2^31 - 1 points");
    }
    for (int c = 0; c < D; ++c) {
        gd.n[c] = g->n[c];
        gd.lo[c] = g->lo[c];
        gd.delta[c] = g->delta[c];
    }
    gd.s[D - 1] = 1;
    for (int c = D - 2; c >= 0; --c) gd.s[c] = gd.s[c + 1] * g->n[c + 1];
    gd.N = (int)N;
    return CVX_OK;
}

template <int D>
int check_dirs(int nd, const int32_t *off, const GridT<D> &gd, std::vector<GridDirT<D>> &dirs,
               std::vector<long long> &line_off) {
    if (nd < 1 || nd > kGridMaxDirs)
        return fail(CVX_ERR_INVALID_ARG, "direction count must be in [1, %d]", kGridMaxDirs);
    if (!off) return fail(CVX_ERR_INVALID_ARG, "direction offsets are NULL");
    constexpr int d = D == 4 ? 2 : 3;
    dirs.resize(nd);
    line_off.assign(nd + 1, 0);
    for (int j = 0; j < nd; ++j) {
        GridDirT<D> g{};
        bool nz = false;
        long long inside = 1;  // points whose predecessor lies in the grid
        for (int c = 0; c < D; ++c) {
            const int o = off[D * j + c];
            if (o < -kGridMaxLine || o > kGridMaxLine)
                return fail(CVX_ERR_INVALID_ARG, "direction %d: offset out of range", j);
            g.o[c] = o;
            nz |= o != 0;
            inside *= std::max(0, gd.n[c] - std::abs(o));
        }
        if (!nz) return fail(CVX_ERR_INVALID_ARG, "direction %d is zero", j);
        // rank one: every 2x2 minor of the d x d offset matrix vanishes
        for (int a = 0; a < d; ++a)
            for (int b = a + 1; b < d; ++b)
                for (int c = 0; c < d; ++c)
                    for (int e = c + 1; e < d; ++e)
                        if ((long long)g.o[d * a + c] * g.o[d * b + e] !=
                            (long long)g.o[d * a + e] * g.o[d * b + c])
                            return fail(CVX_ERR_INVALID_ARG, "direction %d is not rank-one", j);
        long long step = 0;
        for (int c = 0; c < D; ++c) step += (long long)g.o[c] * gd.s[c];
        g.step = (int)step;
        dirs[j] = g;
        line_off[j + 1] = line_off[j] + (gd.N - inside);
    }
    return CVX_OK;
}

// Device buffers shared by cvx_grid_step and cvx_grid_convexify.
template <int D>
struct GridWork {
    GridDirT<D> *dirs;
    long long *line_off;
    unsigned *hist;  // nd x (longest line + 1): line counts, then offsets, by length
    int *starts;
    double *H;
    unsigned *S;
    double *rcp;
    int chunk;  // directions per chunk
};

template <int D>
size_t grid_work_bytes(int nd, const GridT<D> &gd, long long lines, int &chunk) {
    const size_t per_dir = (size_t)gd.N * (sizeof(double) + sizeof(unsigned));
    chunk = (int)std::max<size_t>(1, std::min<size_t>(nd, grid_chunk_bytes() / per_dir));
    return up256(sizeof(GridDirT<D>) * nd) + up256(sizeof(long long) * (nd + 1)) +
           up256(sizeof(unsigned) * nd * (size_t)(kGridMaxLine + 1)) +
           up256(sizeof(int) * (size_t)lines) +
           up256(sizeof(double) * (size_t)chunk * gd.N) +
           up256(sizeof(unsigned) * (size_t)chunk * gd.N) +
           up256(sizeof(double) * (2 * kGridMaxLine + 1));
}

template <int D>
void carve_grid_work(char *ws, int nd, const GridT<D> &gd, long long lines, int chunk,
                     GridWork<D> &w) {
    w.dirs = (GridDirT<D> *)ws;
    ws += up256(sizeof(GridDirT<D>) * nd);
    w.line_off = (long long *)ws;
    ws += up256(sizeof(long long) * (nd + 1));
    w.hist = (unsigned *)ws;
    ws += up256(sizeof(unsigned) * nd * (size_t)(kGridMaxLine + 1));
    w.starts = (int *)ws;
    ws += up256(sizeof(int) * (size_t)lines);
    w.H = (double *)ws;
    ws += up256(sizeof(double) * (size_t)chunk * gd.N);
    w.S = (unsigned *)ws;
    ws += up256(sizeof(unsigned) * (size_t)chunk * gd.N);
    w.rcp = (double *)ws;
    w.chunk = chunk;
}

template <int D>
int grid_line_cap(const GridT<D> &gd) {
    int cap = 1;
    for (int c = 0; c < D; ++c) cap = std::max(cap, gd.n[c]);
    return cap;
}

// Threads per line-kernel CTA so that the stacks fit in shared memory.
int grid_line_threads(int cap) { return cap <= 128 ? 128 : (cap <= 256 ? 64 : 32); }

// Direction table, line regions, line starts and the reciprocal table.
template <int D>
int grid_setup(const GridT<D> &gd, const std::vector<GridDirT<D>> &dirs,
               const std::vector<long long> &line_off, const GridWork<D> &w, cudaStream_t s) {
    const int nd = (int)dirs.size();
    CK(cudaMemcpyAsync(w.dirs, dirs.data(), sizeof(GridDirT<D>) * nd, cudaMemcpyHostToDevice, s),
       "grid setup");
    CK(cudaMemcpyAsync(w.line_off, line_off.data(), sizeof(long long) * (nd + 1),
                       cudaMemcpyHostToDevice, s),
       "grid setup");
    const int cap = grid_line_cap<D>(gd);
    CK(cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * nd * (size_t)(cap + 1), s), "grid setup");
    const size_t smem = sizeof(int) * (size_t)nd * D;
    CK(cudaFuncSetAttribute(k_grid_starts<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem),
       "grid line starts shared memory");
    const int bx = (int)std::min<long long>((gd.N + 255) / 256, 4096);
    k_grid_starts<D><<<bx, 256, smem, s>>>(gd, w.dirs, nd, w.line_off, w.hist, cap, 0, w.starts);
    CK(cudaGetLastError(), "grid line counts");
    k_grid_len_scan<<<(nd + 127) / 128, 128, 0, s>>>(nd, cap, w.hist);
    CK(cudaGetLastError(), "grid line offsets");
    k_grid_starts<D><<<bx, 256, smem, s>>>(gd, w.dirs, nd, w.line_off, w.hist, cap, 1, w.starts);
    CK(cudaGetLastError(), "grid line starts");
    k_grid_rcp<<<(2 * kGridMaxLine + 256) / 256, 256, 0, s>>>(w.rcp);
    CK(cudaGetLastError(), "grid reciprocal table");
    return CVX_OK;
}

// One step (all chunks) from Win to Wout.
template <int D>
int grid_enqueue_step(const GridT<D> &gd, int nd, const std::vector<long long> &line_off,
                      const GridWork<D> &w, int cap, const double *Win, double *Wout, int *lam,
                      unsigned long long *dec, const int *done, cudaStream_t s,
                      cvx_handle *h) {
    const int T = grid_line_threads(cap);
    const size_t smem = (size_t)cap * T * (sizeof(double) + sizeof(short));
    for (int j0 = 0; j0 < nd; j0 += w.chunk) {
        const int j1 = std::min(nd, j0 + w.chunk);
        const long long lines = line_off[j1] - line_off[j0];
        if (lines > 0) {
            std::vector<cudaEvent_t> ev;
            int rc = scan_events(h, 1, ev);
            if (rc) return rc;
            if (!ev.empty()) CK(cudaEventRecord(ev[0], s), "grid profiling");
            k_grid_lines<D><<<(unsigned)((lines + T - 1) / T), T, smem, s>>>(
                gd, w.dirs, w.line_off, j0, j1, w.starts, Win, w.H, w.S, cap, done);
            CK(cudaGetLastError(), "grid line kernel");
            if (!ev.empty()) CK(cudaEventRecord(ev[1], s), "grid profiling");
        }
        k_grid_reduce<<<(gd.N + 255) / 256, 256, 0, s>>>(gd.N, j0, j1, j0 == 0, j1 == nd, Win,
                                                         w.H, w.S, w.rcp, Wout, lam, dec, done);
        CK(cudaGetLastError(), "grid reduce kernel");
    }
    return CVX_OK;
}

template <int D>
int set_line_smem(int cap) {
    const int T = grid_line_threads(cap);
    const size_t smem = (size_t)cap * T * (sizeof(double) + sizeof(short));
    CK(cudaFuncSetAttribute(k_grid_lines<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem),
       "grid line kernel shared memory");
    return CVX_OK;
}

int check_grid_call(const cvx_params *p, const cvx_grid *g, int32_t det_rule, double beta_k) {
    if (p) {
        int rc = check_params(p, false, true);
        if (rc) return rc;
    }
    if (!g) return fail(CVX_ERR_INVALID_ARG, "grid is NULL");
    if (g->dim != 2 && g->dim != 3) return fail(CVX_ERR_INVALID_ARG, "grid dim must be 2 or 3");
    if (p && g->dim == 3 && p->energy == CVX_ENERGY_DOUBLE_WELL)
        return fail(CVX_ERR_INVALID_ARG, "the double-well energy is two-dimensional");
    if (det_rule != 0 && det_rule != 1) return fail(CVX_ERR_INVALID_ARG, "det_rule must be 0 or 1");
    if (!isfinite(beta_k)) return fail(CVX_ERR_INVALID_ARG, "beta_k must be finite");
    return CVX_OK;
}

template <int D>
int grid_energy_t(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                  int32_t rule, double *W, cudaStream_t s) {
    GridT<D> gd;
    int rc = check_grid<D>(g, gd);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W) return fail(CVX_ERR_INVALID_ARG, "W is NULL");
    DeviceGuard dg(h->device);
    k_grid_energy<D><<<(gd.N + 255) / 256, 256, 0, s>>>(gd, material_of(p), beta_k, rule, W);
    CK(cudaGetLastError(), "cvx_grid_energy");
    return CVX_OK;
}

template <int D>
int grid_step_t(cvx_handle *h, const cvx_grid *g, int32_t nd, const int32_t *off,
                const double *W_in, double *W_out, int32_t *lam, double *dec, cudaStream_t s) {
    GridT<D> gd;
    int rc = check_grid<D>(g, gd);
    if (rc) return rc;
    std::vector<GridDirT<D>> dirs;
    std::vector<long long> line_off;
    rc = check_dirs<D>(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W_in || !W_out) return fail(CVX_ERR_INVALID_ARG, "W_in and W_out are required");
    if (W_in == W_out) return fail(CVX_ERR_INVALID_ARG, "W_out must not alias W_in");
    DeviceGuard dg(h->device);
    const long long lines = line_off[nd];
    int chunk = 0;
    size_t bytes = grid_work_bytes<D>(nd, gd, lines, chunk);
    const size_t lam_off = bytes;
    if (!lam) bytes += up256(sizeof(int) * 3 * (size_t)gd.N);
    rc = ensure_ws(h, bytes, s);
    if (rc) return rc;
    GridWork<D> w;
    carve_grid_work<D>(h->ws, nd, gd, lines, chunk, w);
    int *lam_w = lam ? lam : (int *)(h->ws + lam_off);
    const int cap = grid_line_cap<D>(gd);
    rc = set_line_smem<D>(cap);
    if (rc) return rc;
    rc = grid_setup<D>(gd, dirs, line_off, w, s);
    if (rc) return rc;
    if (dec) CK(cudaMemsetAsync(dec, 0, sizeof(double), s), "cvx_grid_step");
    return grid_enqueue_step<D>(gd, nd, line_off, w, cap, W_in, W_out, lam_w,
                                reinterpret_cast<unsigned long long *>(dec), nullptr, s, h);
}

template <int D>
int grid_convexify_t(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                     int32_t rule, int32_t nd, const int32_t *off, int32_t kmax, double tol,
                     double *W, int32_t *forest, double *decs, int32_t *iters, cudaStream_t s) {
    GridT<D> gd;
    int rc = check_grid<D>(g, gd);
    if (rc) return rc;
    std::vector<GridDirT<D>> dirs;
    std::vector<long long> line_off;
    rc = check_dirs<D>(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (kmax < 1 || kmax > kGridMaxIters)
        return fail(CVX_ERR_INVALID_ARG, "kmax must be in [1, %d]", kGridMaxIters);
    if (!(tol >= 0.0)) return fail(CVX_ERR_INVALID_ARG, "tol must be >= 0");
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W || !iters) return fail(CVX_ERR_INVALID_ARG, "W and iters are required");
    DeviceGuard dg(h->device);
    const long long lines = line_off[nd];
    int chunk = 0;
    size_t bytes = grid_work_bytes<D>(nd, gd, lines, chunk);
    const size_t o_pong = bytes;
    bytes += up256(sizeof(double) * (size_t)gd.N);
    const size_t o_lam = bytes;
    if (!forest) bytes += up256(sizeof(int) * 3 * (size_t)gd.N);
    const size_t o_dec = bytes;
    if (!decs) bytes += up256(sizeof(double) * kmax);
    const size_t o_done = bytes;
    bytes += 256;
    rc = ensure_ws(h, bytes, s);
    if (rc) return rc;
    GridWork<D> w;
    carve_grid_work<D>(h->ws, nd, gd, lines, chunk, w);
    double *pong = (double *)(h->ws + o_pong);
    unsigned long long *dk =
        reinterpret_cast<unsigned long long *>(decs ? decs : (double *)(h->ws + o_dec));
    int *done = (int *)(h->ws + o_done);
    const int cap = grid_line_cap<D>(gd);
    rc = set_line_smem<D>(cap);
    if (rc) return rc;
    rc = grid_setup<D>(gd, dirs, line_off, w, s);
    if (rc) return rc;
    CK(cudaMemsetAsync(dk, 0, sizeof(double) * kmax, s), "cvx_grid_convexify");
    CK(cudaMemsetAsync(done, 0, sizeof(int), s), "cvx_grid_convexify");
    CK(cudaMemsetAsync(iters, 0, sizeof(int32_t), s), "cvx_grid_convexify");
    const unsigned pb = (unsigned)((gd.N + 255) / 256);
    k_grid_energy<D><<<pb, 256, 0, s>>>(gd, material_of(p), beta_k, rule, W);
    CK(cudaGetLastError(), "cvx_grid_convexify energy");
    for (int k = 0; k < kmax; ++k) {
        const double *in = (k & 1) ? pong : W;
        double *out = (k & 1) ? W : pong;
        int *lam = forest ? forest + 3 * (size_t)k * gd.N : (int *)(h->ws + o_lam);
        rc = grid_enqueue_step<D>(gd, nd, line_off, w, cap, in, out, lam, dk + k, done, s, h);
        if (rc) return rc;
        k_grid_check<<<1, 1, 0, s>>>(dk + k, tol, done, iters, k);
        CK(cudaGetLastError(), "cvx_grid_convexify check");
    }
    k_grid_final<<<pb, 256, 0, s>>>(gd.N, iters, pong, W);
    CK(cudaGetLastError(), "cvx_grid_convexify final");
    return CVX_OK;
}

template <int D>
int grid_query_t(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                 int32_t rule, int32_t nd, const int32_t *off, int32_t K, const double *WK,
                 const int32_t *forest, int64_t n, const double *F, double *W_interp,
                 double *W_tree, double *P, double *A, int64_t *leaves, cudaStream_t s) {
    GridT<D> gd;
    int rc = check_grid<D>(g, gd);
    if (rc) return rc;
    std::vector<GridDirT<D>> dirs;
    std::vector<long long> line_off;
    rc = check_dirs<D>(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (K < 0 || K > kGridMaxIters)
        return fail(CVX_ERR_INVALID_ARG, "K must be in [0, %d]", kGridMaxIters);
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!WK || !F || !W_interp || !W_tree || !P || (K > 0 && !forest)))
        return fail(CVX_ERR_INVALID_ARG, "NULL array (WK, F, W_interp, W_tree, P; forest if K > 0)");
    if (n == 0) return CVX_OK;
    DeviceGuard dg(h->device);
    // tables: the leaves (order 0) and two buffers of orders, each
    // W[N], P[D][N], leaves[N] (and A[D^2][N] when the tangent is asked for)
    const int na = A ? D * D : 0;
    const size_t tab = up256(sizeof(double) * (D + 1 + na) * (size_t)gd.N) +
                       up256(sizeof(long long) * (size_t)gd.N);
    const size_t o_t = up256(sizeof(GridDirT<D>) * nd);
    rc = ensure_ws(h, o_t + 3 * tab, s);
    if (rc) return rc;
    GridDirT<D> *dd = (GridDirT<D> *)h->ws;
    struct Tab {
        double *w, *p, *a;
        long long *l;
    };
    auto carve = [&](int i) {
        char *b = h->ws + o_t + i * tab;
        Tab t;
        t.w = (double *)b;
        t.p = t.w + gd.N;
        t.a = A ? t.p + (size_t)D * gd.N : nullptr;
        t.l = (long long *)(b + up256(sizeof(double) * (D + 1 + na) * (size_t)gd.N));
        return t;
    };
    const Tab t0 = carve(0), ta = carve(1), tb = carve(2);
    CK(cudaMemcpyAsync(dd, dirs.data(), sizeof(GridDirT<D>) * nd, cudaMemcpyHostToDevice, s),
       "cvx_grid_query");
    const unsigned pbk = (unsigned)((gd.N + 255) / 256);
    k_grid_tree0<D><<<pbk, 256, 0, s>>>(gd, material_of(p), beta_k, rule, t0.w, t0.p, t0.l, t0.a);
    CK(cudaGetLastError(), "cvx_grid_query leaves");
    Tab cur = t0;
    for (int d = 1; d <= K; ++d) {
        const Tab nx = (d & 1) ? ta : tb;
        k_grid_tree_step<D><<<pbk, 256, 0, s>>>(gd, dd, nd, forest + 3 * (size_t)(d - 1) * gd.N,
                                                t0.w, t0.p, t0.l, cur.w, cur.p, cur.l, nx.w, nx.p,
                                                nx.l, t0.a, cur.a, nx.a);
        CK(cudaGetLastError(), "cvx_grid_query tree order");
        cur = nx;
    }
    k_grid_query<D><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
        gd, WK, cur.w, cur.p, cur.l, cur.a, n, F, W_interp, W_tree, P, A,
        reinterpret_cast<long long *>(leaves));
    CK(cudaGetLastError(), "cvx_grid_query");
    return CVX_OK;
}

}  // namespace
}  // namespace cvx

using namespace cvx;

extern "C" {

int cvx_grid_r11(int32_t dim, int32_t *off) {
    if (!off) return fail(CVX_ERR_INVALID_ARG, "off is NULL");
    if (dim == 2) {
        // a, b over (1,0), (0,1), (1,1), (1,-1): one of each pair +-v (the
        // sign of a (x) b gives the same line); direction 4 ia + ib
        static const int v[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
        for (int ia = 0; ia < 4; ++ia)
            for (int ib = 0; ib < 4; ++ib)
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j)
                        off[4 * (4 * ia + ib) + 2 * i + j] = v[ia][i] * v[ib][j];
        return CVX_OK;
    }
    if (dim == 3) {
        // the 13 vectors of {-1,0,1}^3 with first nonzero entry +1: axes,
        // face diagonals, body diagonals; direction 13 ia + ib
        static const int v[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                     {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                     {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
        for (int ia = 0; ia < 13; ++ia)
            for (int ib = 0; ib < 13; ++ib)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        off[9 * (13 * ia + ib) + 3 * i + j] = v[ia][i] * v[ib][j];
        return CVX_OK;
    }
    return fail(CVX_ERR_INVALID_ARG, "dim must be 2 or 3");
}

int cvx_grid_energy(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                    int32_t det_rule, double *W, cvx_stream sv) {
    if (!p) return fail(CVX_ERR_INVALID_ARG, "params is NULL");
    int rc = check_grid_call(p, g, det_rule, beta_k);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)sv;
    return g->dim == 2 ? grid_energy_t<4>(h, p, g, beta_k, det_rule, W, s)
                       : grid_energy_t<9>(h, p, g, beta_k, det_rule, W, s);
}

int cvx_grid_step(cvx_handle *h, const cvx_grid *g, int32_t nd, const int32_t *off,
                  const double *W_in, double *W_out, int32_t *lam, double *dec, cvx_stream sv) {
    int rc = check_grid_call(nullptr, g, 0, 0.0);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)sv;
    return g->dim == 2 ? grid_step_t<4>(h, g, nd, off, W_in, W_out, lam, dec, s)
                       : grid_step_t<9>(h, g, nd, off, W_in, W_out, lam, dec, s);
}

int cvx_grid_convexify(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                       int32_t det_rule, int32_t nd, const int32_t *off, int32_t kmax, double tol,
                       double *W, int32_t *forest, double *decs, int32_t *iters,
                       cvx_stream sv) {
    if (!p) return fail(CVX_ERR_INVALID_ARG, "params is NULL");
    int rc = check_grid_call(p, g, det_rule, beta_k);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)sv;
    return g->dim == 2 ? grid_convexify_t<4>(h, p, g, beta_k, det_rule, nd, off, kmax, tol, W,
                                             forest, decs, iters, s)
                       : grid_convexify_t<9>(h, p, g, beta_k, det_rule, nd, off, kmax, tol, W,
                                             forest, decs, iters, s);
}

int cvx_grid_query(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                   int32_t det_rule, int32_t nd, const int32_t *off, int32_t K, const double *WK,
                   const int32_t *forest, int64_t n, const double *F, double *W_interp,
                   double *W_tree, double *P, double *A, int64_t *leaves, cvx_stream sv) {
    if (!p) return fail(CVX_ERR_INVALID_ARG, "params is NULL");
    int rc = check_grid_call(p, g, det_rule, beta_k);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)sv;
    return g->dim == 2 ? grid_query_t<4>(h, p, g, beta_k, det_rule, nd, off, K, WK, forest, n, F,
                                         W_interp, W_tree, P, A, leaves, s)
                       : grid_query_t<9>(h, p, g, beta_k, det_rule, nd, off, K, WK, forest, n, F,
                                         W_interp, W_tree, P, A, leaves, s);
}

}  // extern "C"
