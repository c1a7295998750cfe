// cvx_grid.cu -- the global-grid form of the method (Secs. 4.1-4.3, 5.1-5.3):
// Eq. (4.3) iterated on the cuboid deformation-gradient grid of Sec. 5.2 with
// a set of grid-index directions (the reduced set R^1_1 of Eq. 5.1), the
// one-dimensional convexification of Algorithm 1 on every rank-one line of
// the grid, the lamination forest, and Algorithm 2's trees (with the
// multilinear-interpolation branching of Sec. 5.3) evaluated by Algorithm 3
// at arbitrary points.
//
// Design.  For a direction R every grid point lies on exactly one maximal
// line {F + l R} of the grid, and all points of one line share the line's
// lower hull: the value of Eq. (4.3) at a point is the hull read at that
// point.  So one thread builds Algorithm 1's hull of one (direction, line)
// pair once (a stack in shared memory) and then walks the line again, reading
// the chord of the hull edge over every point.  The per-point minimum over
// the directions (lowest direction index on equal values, a strict decrease
// required) is a second kernel over the points.  Predicates and chord values
// are the FP64 expressions of the hull at the point with every operation
// rounded on its own (no contraction into FMA): the hull's vertex set does not
// depend on where the line is read, so each step is reproducible bit for bit.
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
constexpr size_t kGridChunkBytes = (size_t)512 << 20;  // per-direction line results per chunk

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

struct GridDev {
    int n[4];
    int s[4];  // flat-index strides (F22 fastest)
    double lo[4], delta[4];
    int N;
};

struct GridDir {
    int o[4];  // grid-index offset of one step along the line
    int step;  // its flat-index step
    int pad;
};

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

__device__ __forceinline__ void grid_index(const GridDev &g, int idx, int i[4]) {
    for (int c = 3; c >= 0; --c) {
        i[c] = idx % g.n[c];
        idx /= g.n[c];
    }
}

// Grid point F_c = lo_c + i_c delta_c, each operation rounded on its own.
__device__ __forceinline__ void grid_point(const GridDev &g, int idx, double F[4]) {
    int i[4];
    grid_index(g, idx, i);
    for (int c = 0; c < 4; ++c) F[c] = __dadd_rn(g.lo[c], __dmul_rn((double)i[c], g.delta[c]));
}

// Energy of the grid study.  abs_det = 0: Eq. (2.9) with det F <= 0 excluded
// (NaN).  abs_det = 1: the Neo-Hooke energy takes ln|det F|, so that a point
// with det F < 0 mirrors one with det F > 0 (only det F = 0 is excluded).
__device__ double grid_w64(const double F[4], double beta, const Material &m, int abs_det) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL || !abs_det) return energy64(F, beta, m);
    const double J = fabs(F[0] * F[3] - F[1] * F[2]);
    if (!(J > 0.0)) return nan("");
    const double lj = log(J);
    const double i1 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3] + 1.0;
    const double s = 0.5 * m.mu * (i1 - 3.0) - m.mu * lj + 0.5 * m.lam * lj * lj;
    const double ek = exp(-beta / m.D0);
    if (s <= beta) return (1.0 - m.Dinf * (1.0 - ek)) * (s - beta);
    return (1.0 - m.Dinf) * (s - beta) + m.Dinf * m.D0 * (ek - exp(-s / m.D0));
}

// dW/dF of grid_w64: (1 - D(max(s, beta))) (mu F - mu F^-T + lambda ln|J| F^-T);
// d ln|J| / dF = F^-T for either sign of J.
__device__ void grid_p64(const double F[4], double beta, const Material &m, int abs_det,
                         double P[4]) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL || !abs_det) {
        stress64(F, beta, m, P);
        return;
    }
    const double J = F[0] * F[3] - F[1] * F[2];
    if (!(fabs(J) > 0.0)) {
        P[0] = P[1] = P[2] = P[3] = nan("");
        return;
    }
    const double lj = log(fabs(J));
    const double i1 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3] + 1.0;
    const double s = 0.5 * m.mu * (i1 - 3.0) - m.mu * lj + 0.5 * m.lam * lj * lj;
    const double b = s > beta ? s : beta;
    const double gd = 1.0 - m.Dinf * (1.0 - exp(-b / m.D0));
    const double FiT[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};
    for (int k = 0; k < 4; ++k) P[k] = gd * (m.mu * F[k] - m.mu * FiT[k] + m.lam * lj * FiT[k]);
}

// Number of grid points on the line that starts at index i along offset o.
__device__ __forceinline__ int line_length(const GridDev &g, const int i[4], const int o[4]) {
    int len = 1 << 30;
    for (int c = 0; c < 4; ++c) {
        if (o[c] > 0) len = min(len, (g.n[c] - 1 - i[c]) / o[c]);
        else if (o[c] < 0) len = min(len, i[c] / (-o[c]));
    }
    return len + 1;
}

// W^0 on the grid.
__global__ void k_grid_energy(GridDev g, Material m, double beta, int abs_det, double *W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    double F[4];
    grid_point(g, p, F);
    W[p] = grid_w64(F, beta, m, abs_det);
}

// Line starts: the points whose predecessor along direction j lies outside the
// grid, written to region j of `starts` (line_off[j] .. line_off[j + 1]).
// Within a warp the order of the points is kept.
__global__ void k_grid_starts(GridDev g, const GridDir *dirs, const long long *line_off,
                              unsigned *fill, int *starts) {
    const int j = blockIdx.y;
    const GridDir d = dirs[j];
    const int lane = threadIdx.x & 31;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < g.N;
         b += (long long)gridDim.x * blockDim.x) {
        const long long p = b + threadIdx.x;
        bool st = false;
        if (p < g.N) {
            int i[4];
            grid_index(g, (int)p, i);
            for (int c = 0; c < 4; ++c) {
                const int q = i[c] - d.o[c];
                st |= (q < 0) || (q >= g.n[c]);
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, st);
        unsigned base = 0;
        if (lane == 0 && mask) base = atomicAdd(&fill[j], (unsigned)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (st) starts[line_off[j] + base + __popc(mask & ((1u << lane) - 1))] = (int)p;
    }
}

// One thread per (direction, line) of directions [j0, j1): Algorithm 1 on the
// finite values of W_in along the line (stack in shared memory, layout
// [slot][thread]), then every point of the line reads the hull there:
//   a hull vertex keeps its own value (no split, S = 0);
//   a point strictly between vertices a < x < b gets the chord value
//   h = (x_b w_a - x_a w_b) / (x_b - x_a) with x_a, x_b taken relative to the
//   point (x_a < 0 < x_b), and S = the pair (x_a, x_b) as two 16-bit fields.
// Non-finite points keep their value.  H and S are chunk-major: entry
// (j - j0) N + point.
__global__ void __launch_bounds__(128) k_grid_lines(GridDev g, const GridDir *dirs,
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
    const GridDir d = dirs[j];
    const int p0 = starts[t];
    int i0[4];
    grid_index(g, p0, i0);
    const int len = line_length(g, i0, d.o);
    double *sv = gsm + threadIdx.x;
    short *sx = reinterpret_cast<short *>(gsm + (size_t)cap * T) + threadIdx.x;

    // Algorithm 1: monotone chain over the finite values, pops while the top
    // of the stack is not strictly below the chord to the new point
    int k = 0;
    for (int l = 0; l < len; ++l) {
        const double w = Win[p0 + l * d.step];
        if (!isfinite(w)) continue;
        while (k >= 2) {
            const double wp = sv[(k - 2) * T], wq = sv[(k - 1) * T];
            const int xp = sx[(k - 2) * T], xq = sx[(k - 1) * T];
            const double A = __dsub_rn(wq, wp), B = __dsub_rn(w, wq);
            const int di = l - xq, dp = xq - xp;
            // multiplying by 1 is exact: skip it
            const double lhs = di == 1 ? A : __dmul_rn(A, exact_double(di));
            const double rhs = dp == 1 ? B : __dmul_rn(B, exact_double(dp));
            if (lhs >= rhs) --k;
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
        const double w0 = Win[idx];
        double hv = w0;
        unsigned sp = 0;
        if (isfinite(w0)) {
            while (e + 1 < k && sx[(e + 1) * T] <= l) ++e;
            const int xa = sx[e * T];
            if (xa != l) {
                const int ra = xa - l, rb = sx[(e + 1) * T] - l;
                const double num = __dsub_rn(__dmul_rn(exact_double(rb), sv[e * T]),
                                             __dmul_rn(exact_double(ra), sv[(e + 1) * T]));
                hv = __ddiv_rn(num, exact_double(rb - ra));
                sp = ((unsigned)ra & 0xffffu) | ((unsigned)rb << 16);
            }
        }
        H[base + idx] = hv;
        S[base + idx] = sp;
    }
}

// Per point, directions [j0, j1) in order: the first strict decrease below
// the best so far wins (first chunk: the best so far is W_in itself, no
// split).  lam = (dir, l-, l+) per point (dir = -1: no split).  The last
// chunk adds the point's decrease W_in - W_out to the step's maximum (dec,
// as the bits of a non-negative double).
__global__ void k_grid_reduce(int N, int j0, int j1, int first, int last, const double *Win,
                              const double *H, const unsigned *S, double *Wout, int *lam,
                              unsigned long long *dec, const int *done) {
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
                const double h = H[e];
                if (h < best) {
                    best = h;
                    bd = j;
                    bm = (int)(short)(s & 0xffffu);
                    bp = (int)(s >> 16);
                }
            }
        }
        Wout[p] = best;
        lam[3 * p] = bd;
        lam[3 * p + 1] = bm;
        lam[3 * p + 2] = bp;
        if (last && isfinite(w0) && isfinite(best))
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

// Interpolation decomposition (Sec. 5.3): the corners of the grid cell that
// holds F with their multilinear weights; a coordinate within 1e-12 of a grid
// value counts as on it, corners of weight 0 are left out.  Returns the
// number of corners (0 outside the grid).
__device__ int grid_decompose(const GridDev &g, const double F[4], int cidx[16], double cw[16]) {
    int i0[4];
    double t[4];
    for (int c = 0; c < 4; ++c) {
        const double u = __ddiv_rn(__dsub_rn(F[c], g.lo[c]), g.delta[c]);
        if (u < -1e-12 || u > (double)(g.n[c] - 1) + 1e-12) return 0;
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
    int nc = 0;
    for (int corner = 0; corner < 16; ++corner) {
        double w = 1.0;
        int flat = 0;
        for (int c = 0; c < 4; ++c) {
            const int up = (corner >> (3 - c)) & 1;
            w = __dmul_rn(w, up ? t[c] : __dsub_rn(1.0, t[c]));
            flat += (i0[c] + up) * g.s[c];
        }
        if (w == 0.0) continue;
        cidx[nc] = flat;
        cw[nc] = w;
        ++nc;
    }
    return nc;
}

// Algorithm 2's tree at n points evaluated by Algorithm 3, one thread per
// point: the interpolation corners at order K, each expanded depth first
// through the forest (the latest iteration k <= d that split a grid point
// gives its children F- (weight 1 - xi) then F+ (weight xi) at order k - 1,
// xi = -l- / (l+ - l-)); leaves add weight (W, P).  W_interp is the
// multilinear interpolation of W^K.  Sums run in the order of the recursion.
__global__ void k_grid_query(GridDev g, Material m, double beta, int abs_det,
                             const GridDir *dirs, int nd, int K, const double *WK,
                             const int *forest,
                             long long n, const double *F, double *Wi, double *Wt, double *P,
                             long long *leaves) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double G[4] = {F[4 * q], F[4 * q + 1], F[4 * q + 2], F[4 * q + 3]};
    int cidx[16];
    double cw[16];
    const int nc = grid_decompose(g, G, cidx, cw);
    double wi = 0.0, wt = 0.0, Pp[4] = {0.0, 0.0, 0.0, 0.0};
    long long nl = 0;
    int st_idx[kGridMaxIters + 2], st_d[kGridMaxIters + 2];
    double st_w[kGridMaxIters + 2];
    for (int c = 0; c < nc; ++c) {
        wi = __dadd_rn(wi, __dmul_rn(cw[c], WK[cidx[c]]));
        int sp = 0;
        st_idx[0] = cidx[c];
        st_d[0] = K;
        st_w[0] = cw[c];
        sp = 1;
        while (sp > 0) {
            --sp;
            const int idx = st_idx[sp];
            const double wgt = st_w[sp];
            int k = st_d[sp];
            while (k >= 1 && forest[3 * ((long long)(k - 1) * g.N + idx)] < 0) --k;
            if (k < 1) {
                double Fl[4], Pl[4];
                grid_point(g, idx, Fl);
                wt = __dadd_rn(wt, __dmul_rn(wgt, grid_w64(Fl, beta, m, abs_det)));
                grid_p64(Fl, beta, m, abs_det, Pl);
                for (int a = 0; a < 4; ++a) Pp[a] = __dadd_rn(Pp[a], __dmul_rn(wgt, Pl[a]));
                ++nl;
                continue;
            }
            const int *lam = forest + 3 * ((long long)(k - 1) * g.N + idx);
            const int dj = lam[0], lm = lam[1], lp = lam[2];
            const long long cm = idx + (long long)lm * (dj < nd ? dirs[dj].step : 0);
            const long long cp = idx + (long long)lp * (dj < nd ? dirs[dj].step : 0);
            if (dj >= nd || !(lm < 0 && lp > 0) || cm < 0 || cm >= g.N || cp < 0 || cp >= g.N) {
                // not a record this library writes: the point counts as a leaf
                double Fl[4], Pl[4];
                grid_point(g, idx, Fl);
                wt = __dadd_rn(wt, __dmul_rn(wgt, grid_w64(Fl, beta, m, abs_det)));
                grid_p64(Fl, beta, m, abs_det, Pl);
                for (int a = 0; a < 4; ++a) Pp[a] = __dadd_rn(Pp[a], __dmul_rn(wgt, Pl[a]));
                ++nl;
                continue;
            }
            const double xi = __ddiv_rn((double)(-lm), (double)(lp - lm));
            // F+ below F-, so that F- is expanded first
            st_idx[sp] = (int)cp;
            st_d[sp] = k - 1;
            st_w[sp] = __dmul_rn(wgt, xi);
            ++sp;
            st_idx[sp] = (int)cm;
            st_d[sp] = k - 1;
            st_w[sp] = __dmul_rn(wgt, __dsub_rn(1.0, xi));
            ++sp;
        }
    }
    if (nc == 0) wi = wt = Pp[0] = Pp[1] = Pp[2] = Pp[3] = nan("");
    Wi[q] = wi;
    Wt[q] = wt;
    for (int a = 0; a < 4; ++a) P[4 * q + a] = Pp[a];
    if (leaves) leaves[q] = nl;
}

// ------------------------------------------------------------------ host

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_grid(const cvx_grid *g, GridDev &gd) {
    if (!g) return fail(CVX_ERR_INVALID_ARG, "grid is NULL");
    long long N = 1;
    for (int c = 0; c < 4; ++c) {
        if (g->n[c] < 1 || g->n[c] > kGridMaxLine)
            return fail(CVX_ERR_INVALID_ARG, "grid points per component must be in [1, %d]",
                        kGridMaxLine);
        if (!(g->delta[c] > 0.0) || !isfinite(g->delta[c]) || !isfinite(g->lo[c]))
            return fail(CVX_ERR_INVALID_ARG, "grid spacing must be positive and bounds finite");
        N *= g->n[c];
    }
    if (N > 0x7fffffffLL) return fail(CVX_ERR_INVALID_ARG, "grid has more than 2^31 - 1 points");
    for (int c = 0; c < 4; ++c) {
        gd.n[c] = g->n[c];
        gd.lo[c] = g->lo[c];
        gd.delta[c] = g->delta[c];
    }
    gd.s[3] = 1;
    for (int c = 2; c >= 0; --c) gd.s[c] = gd.s[c + 1] * g->n[c + 1];
    gd.N = (int)N;
    return CVX_OK;
}

int check_dirs(int nd, const int32_t *off, const GridDev &gd, std::vector<GridDir> &dirs,
               std::vector<long long> &line_off) {
    if (nd < 1 || nd > kGridMaxDirs)
        return fail(CVX_ERR_INVALID_ARG, "direction count must be in [1, %d]", kGridMaxDirs);
    if (!off) return fail(CVX_ERR_INVALID_ARG, "direction offsets are NULL");
    dirs.resize(nd);
    line_off.assign(nd + 1, 0);
    for (int j = 0; j < nd; ++j) {
        GridDir d{};
        bool nz = false;
        long long inside = 1;  // points whose predecessor lies in the grid
        for (int c = 0; c < 4; ++c) {
            const int o = off[4 * j + c];
            if (o < -kGridMaxLine || o > kGridMaxLine)
                return fail(CVX_ERR_INVALID_ARG, "direction %d: offset out of range", j);
            d.o[c] = o;
            nz |= o != 0;
            inside *= std::max(0, gd.n[c] - std::abs(o));
        }
        if (!nz) return fail(CVX_ERR_INVALID_ARG, "direction %d is zero", j);
        if ((long long)d.o[0] * d.o[3] != (long long)d.o[1] * d.o[2])
            return fail(CVX_ERR_INVALID_ARG, "direction %d is not rank-one", j);
        d.step = d.o[0] * gd.s[0] + d.o[1] * gd.s[1] + d.o[2] * gd.s[2] + d.o[3] * gd.s[3];
        dirs[j] = d;
        line_off[j + 1] = line_off[j] + (gd.N - inside);
    }
    return CVX_OK;
}

// Device buffers shared by cvx_grid_step and cvx_grid_convexify.
struct GridWork {
    GridDir *dirs;
    long long *line_off;
    unsigned *fill;
    int *starts;
    double *H;
    unsigned *S;
    int chunk;  // directions per chunk
};

size_t grid_work_bytes(int nd, const GridDev &gd, long long lines, int &chunk) {
    const size_t per_dir = (size_t)gd.N * (sizeof(double) + sizeof(unsigned));
    chunk = (int)std::max<size_t>(1, std::min<size_t>(nd, grid_chunk_bytes() / per_dir));
    return up256(sizeof(GridDir) * nd) + up256(sizeof(long long) * (nd + 1)) +
           up256(sizeof(unsigned) * nd) + up256(sizeof(int) * (size_t)lines) +
           up256(sizeof(double) * (size_t)chunk * gd.N) +
           up256(sizeof(unsigned) * (size_t)chunk * gd.N);
}

char *carve_grid_work(char *ws, int nd, const GridDev &gd, long long lines, int chunk,
                      GridWork &w) {
    w.dirs = (GridDir *)ws;
    ws += up256(sizeof(GridDir) * nd);
    w.line_off = (long long *)ws;
    ws += up256(sizeof(long long) * (nd + 1));
    w.fill = (unsigned *)ws;
    ws += up256(sizeof(unsigned) * nd);
    w.starts = (int *)ws;
    ws += up256(sizeof(int) * (size_t)lines);
    w.H = (double *)ws;
    ws += up256(sizeof(double) * (size_t)chunk * gd.N);
    w.S = (unsigned *)ws;
    ws += up256(sizeof(unsigned) * (size_t)chunk * gd.N);
    w.chunk = chunk;
    return ws;
}

int grid_line_cap(const GridDev &gd) {
    int cap = 1;
    for (int c = 0; c < 4; ++c) cap = std::max(cap, gd.n[c]);
    return cap;
}

// Threads per line-kernel CTA so that the stacks fit in shared memory.
int grid_line_threads(int cap) { return cap <= 128 ? 128 : (cap <= 256 ? 64 : 32); }

// Direction table, line regions and line starts of one call.
int grid_setup(const GridDev &gd, const std::vector<GridDir> &dirs,
               const std::vector<long long> &line_off, const GridWork &w, cudaStream_t s) {
    const int nd = (int)dirs.size();
    CK(cudaMemcpyAsync(w.dirs, dirs.data(), sizeof(GridDir) * nd, cudaMemcpyHostToDevice, s),
       "grid setup");
    CK(cudaMemcpyAsync(w.line_off, line_off.data(), sizeof(long long) * (nd + 1),
                       cudaMemcpyHostToDevice, s),
       "grid setup");
    CK(cudaMemsetAsync(w.fill, 0, sizeof(unsigned) * nd, s), "grid setup");
    const int bx = (int)std::min<long long>((gd.N + 255) / 256, 1024);
    k_grid_starts<<<dim3(bx, nd), 256, 0, s>>>(gd, w.dirs, w.line_off, w.fill, w.starts);
    CK(cudaGetLastError(), "grid line starts");
    return CVX_OK;
}

// One step (all chunks) from Win to Wout.
int grid_enqueue_step(const GridDev &gd, int nd, const std::vector<long long> &line_off,
                      const GridWork &w, int cap, const double *Win, double *Wout, int *lam,
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
            k_grid_lines<<<(unsigned)((lines + T - 1) / T), T, smem, s>>>(
                gd, w.dirs, w.line_off, j0, j1, w.starts, Win, w.H, w.S, cap, done);
            CK(cudaGetLastError(), "grid line kernel");
            if (!ev.empty()) CK(cudaEventRecord(ev[1], s), "grid profiling");
        }
        k_grid_reduce<<<(gd.N + 255) / 256, 256, 0, s>>>(gd.N, j0, j1, j0 == 0, j1 == nd, Win,
                                                         w.H, w.S, Wout, lam, dec, done);
        CK(cudaGetLastError(), "grid reduce kernel");
    }
    return CVX_OK;
}

int set_line_smem(int cap) {
    const int T = grid_line_threads(cap);
    const size_t smem = (size_t)cap * T * (sizeof(double) + sizeof(short));
    CK(cudaFuncSetAttribute(k_grid_lines, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem),
       "grid line kernel shared memory");
    return CVX_OK;
}

}  // namespace
}  // namespace cvx

using namespace cvx;

extern "C" {

int cvx_grid_r11(int32_t *off) {
    if (!off) return fail(CVX_ERR_INVALID_ARG, "off is NULL");
    // a, b over (1,0), (0,1), (1,1), (1,-1): one of each pair +-v (the sign of
    // a (x) b gives the same line); direction 4 ia + ib, offset
    // (a1 b1, a1 b2, a2 b1, a2 b2) in grid steps
    static const int v[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
    for (int ia = 0; ia < 4; ++ia)
        for (int ib = 0; ib < 4; ++ib) {
            int32_t *o = off + 4 * (4 * ia + ib);
            o[0] = v[ia][0] * v[ib][0];
            o[1] = v[ia][0] * v[ib][1];
            o[2] = v[ia][1] * v[ib][0];
            o[3] = v[ia][1] * v[ib][1];
        }
    return CVX_OK;
}

int cvx_grid_energy(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                    int32_t abs_det, double *W, cvx_stream sv) {
    int rc = check_params(p, false);
    if (rc) return rc;
    GridDev gd;
    rc = check_grid(g, gd);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W) return fail(CVX_ERR_INVALID_ARG, "W is NULL");
    if (!isfinite(beta_k)) return fail(CVX_ERR_INVALID_ARG, "beta_k must be finite");
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    k_grid_energy<<<(gd.N + 255) / 256, 256, 0, s>>>(gd, material_of(p), beta_k, abs_det ? 1 : 0,
                                                      W);
    CK(cudaGetLastError(), "cvx_grid_energy");
    return CVX_OK;
}

int cvx_grid_step(cvx_handle *h, const cvx_grid *g, int32_t nd, const int32_t *off,
                  const double *W_in, double *W_out, int32_t *lam, double *dec, cvx_stream sv) {
    GridDev gd;
    int rc = check_grid(g, gd);
    if (rc) return rc;
    std::vector<GridDir> dirs;
    std::vector<long long> line_off;
    rc = check_dirs(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W_in || !W_out) return fail(CVX_ERR_INVALID_ARG, "W_in and W_out are required");
    if (W_in == W_out) return fail(CVX_ERR_INVALID_ARG, "W_out must not alias W_in");
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    const long long lines = line_off[nd];
    int chunk = 0;
    size_t bytes = grid_work_bytes(nd, gd, lines, chunk);
    const size_t lam_off = bytes;
    if (!lam) bytes += up256(sizeof(int) * 3 * (size_t)gd.N);
    rc = ensure_ws(h, bytes, s);
    if (rc) return rc;
    GridWork w;
    char *tail = carve_grid_work(h->ws, nd, gd, lines, chunk, w);
    (void)tail;
    int *lam_w = lam ? lam : (int *)(h->ws + lam_off);
    const int cap = grid_line_cap(gd);
    rc = set_line_smem(cap);
    if (rc) return rc;
    rc = grid_setup(gd, dirs, line_off, w, s);
    if (rc) return rc;
    if (dec) CK(cudaMemsetAsync(dec, 0, sizeof(double), s), "cvx_grid_step");
    return grid_enqueue_step(gd, nd, line_off, w, cap, W_in, W_out, lam_w,
                             reinterpret_cast<unsigned long long *>(dec), nullptr, s, h);
}

int cvx_grid_convexify(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                       int32_t abs_det, int32_t nd, const int32_t *off, int32_t kmax, double tol,
                       double *W, int32_t *forest, double *decs, int32_t *iters,
                       cvx_stream sv) {
    int rc = check_params(p, false);
    if (rc) return rc;
    GridDev gd;
    rc = check_grid(g, gd);
    if (rc) return rc;
    std::vector<GridDir> dirs;
    std::vector<long long> line_off;
    rc = check_dirs(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (kmax < 1 || kmax > kGridMaxIters)
        return fail(CVX_ERR_INVALID_ARG, "kmax must be in [1, %d]", kGridMaxIters);
    if (!(tol >= 0.0)) return fail(CVX_ERR_INVALID_ARG, "tol must be >= 0");
    if (!isfinite(beta_k)) return fail(CVX_ERR_INVALID_ARG, "beta_k must be finite");
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (!W || !iters) return fail(CVX_ERR_INVALID_ARG, "W and iters are required");
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    const long long lines = line_off[nd];
    int chunk = 0;
    size_t bytes = grid_work_bytes(nd, gd, lines, chunk);
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
    GridWork w;
    carve_grid_work(h->ws, nd, gd, lines, chunk, w);
    double *pong = (double *)(h->ws + o_pong);
    unsigned long long *dk =
        reinterpret_cast<unsigned long long *>(decs ? decs : (double *)(h->ws + o_dec));
    int *done = (int *)(h->ws + o_done);
    const int cap = grid_line_cap(gd);
    rc = set_line_smem(cap);
    if (rc) return rc;
    rc = grid_setup(gd, dirs, line_off, w, s);
    if (rc) return rc;
    CK(cudaMemsetAsync(dk, 0, sizeof(double) * kmax, s), "cvx_grid_convexify");
    CK(cudaMemsetAsync(done, 0, sizeof(int), s), "cvx_grid_convexify");
    CK(cudaMemsetAsync(iters, 0, sizeof(int32_t), s), "cvx_grid_convexify");
    const unsigned pb = (unsigned)((gd.N + 255) / 256);
    k_grid_energy<<<pb, 256, 0, s>>>(gd, material_of(p), beta_k, abs_det ? 1 : 0, W);
    CK(cudaGetLastError(), "cvx_grid_convexify energy");
    for (int k = 0; k < kmax; ++k) {
        const double *in = (k & 1) ? pong : W;
        double *out = (k & 1) ? W : pong;
        int *lam = forest ? forest + 3 * (size_t)k * gd.N : (int *)(h->ws + o_lam);
        rc = grid_enqueue_step(gd, nd, line_off, w, cap, in, out, lam, dk + k, done, s, h);
        if (rc) return rc;
        k_grid_check<<<1, 1, 0, s>>>(dk + k, tol, done, iters, k);
        CK(cudaGetLastError(), "cvx_grid_convexify check");
    }
    k_grid_final<<<pb, 256, 0, s>>>(gd.N, iters, pong, W);
    CK(cudaGetLastError(), "cvx_grid_convexify final");
    return CVX_OK;
}

int cvx_grid_query(cvx_handle *h, const cvx_params *p, const cvx_grid *g, double beta_k,
                   int32_t abs_det, int32_t nd, const int32_t *off, int32_t K, const double *WK,
                   const int32_t *forest, int64_t n, const double *F, double *W_interp,
                   double *W_tree, double *P, int64_t *leaves, cvx_stream sv) {
    int rc = check_params(p, false);
    if (rc) return rc;
    GridDev gd;
    rc = check_grid(g, gd);
    if (rc) return rc;
    std::vector<GridDir> dirs;
    std::vector<long long> line_off;
    rc = check_dirs(nd, off, gd, dirs, line_off);
    if (rc) return rc;
    if (K < 0 || K > kGridMaxIters)
        return fail(CVX_ERR_INVALID_ARG, "K must be in [0, %d]", kGridMaxIters);
    if (!isfinite(beta_k)) return fail(CVX_ERR_INVALID_ARG, "beta_k must be finite");
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!WK || !F || !W_interp || !W_tree || !P || (K > 0 && !forest)))
        return fail(CVX_ERR_INVALID_ARG, "NULL array (WK, F, W_interp, W_tree, P; forest if K > 0)");
    if (n == 0) return CVX_OK;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    const size_t bytes = up256(sizeof(GridDir) * nd);
    rc = ensure_ws(h, bytes, s);
    if (rc) return rc;
    GridDir *dd = (GridDir *)h->ws;
    CK(cudaMemcpyAsync(dd, dirs.data(), sizeof(GridDir) * nd, cudaMemcpyHostToDevice, s),
       "cvx_grid_query");
    k_grid_query<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
        gd, material_of(p), beta_k, abs_det ? 1 : 0, dd, nd, K, WK, forest, n, F, W_interp, W_tree,
        P, reinterpret_cast<long long *>(leaves));
    CK(cudaGetLastError(), "cvx_grid_query");
    return CVX_OK;
}

}  // extern "C"
