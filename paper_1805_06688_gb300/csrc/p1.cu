// The paper's P1-triangle operator (Sec. 2) on the device, FP64: its matrices, the operator
// M_h + s K applied to a batch of slices, the step solve by preconditioned conjugate gradients, and
// the space-time residual of Eq. (3.1) with it.
//
// With U[j][i] = u(x_i, y_j) the printed block forms read
//     (A_x U)[j, :] = c_x ( A_1 U[j, :] + A_2 U[j+1, :] + A_2^T U[j-1, :] )   (blocks over y-lines),
//     (A_y U)[:, i] = c_y ( A_1 U[:, i] + A_2 U[:, i+1] + A_2^T U[:, i-1] )   (the permutation P_pi),
//     (M_h U)[j][i] = h_x h_y / 12 ( 6 U[j][i] + U[j][i-1] + U[j][i+1] + U[j+1][i] + U[j+1][i+1]
//                                    + U[j-1][i] + U[j-1][i-1] ),
// so each stiffness is ONE dense product with the contraction over three shifted copies of U
// (K = 3 P): K_x U = [U | U_{j+1} | U_{j-1}] [A_1; A_2^T; A_2] and K_y U = [A_1 | A_2 | A_2^T]
// [U; U_{i+1}; U_{i-1}].  The shifted copies are never stored: the tile loader reads U at the
// shifted row or column.  The second product's epilogue adds the first one, the 7-point mass
// stencil, the load and the combination the caller asks for, so M_h U + s K U costs two launches.
//
// The step S_n X = R (S_n = M_h + tau_n K, symmetric positive definite by Lemma 3.2) is solved by
// CG preconditioned with the tensor-product operator's fast-diagonalisation solve at the same tau
// (spectrally equivalent: the preconditioned spectrum lies in [0.75, 3] for the paper's orders,
// independent of h and tau), to a relative residual of 1e-13 per slice (the paper solves with CG to
// 1e-9).  Inside MGRIT each solve starts from the value the iterate already holds at its time point
// (the value a relaxation replaces, or the C-point value a residual is taken against): once the
// iteration converges that is close to the step's result and CG needs few iterations; other solves
// start from zero.  Every slice of a batch has its own CG scalars; the iteration stops when the
// slowest slice has converged.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sfde_internal.cuh"

struct SfdeP1 {
    double* Bx = nullptr;     // 3 Px x Px, rows [A_1; A_2^T; A_2] of the x direction (zero padded)
    double* By = nullptr;     // Py x 3 Py, columns [A_1 | A_2 | A_2^T] of the y direction
    double cx = 0, cy = 0;    // the printed prefactors of A_x^beta and A_y^gamma
    double hx = 0, hy = 0;
    size_t ws_slices = 0;
    double* ws = nullptr;     // 7 x ws_slices x P^2: R, X, r, z, p, q, T
    double* dots = nullptr;   // 6 x ws_slices per-slice scalars
    double* hmax = nullptr;   // pinned host scalar
    int last_iters = 0;       // CG iterations of the last step batch
    long long total_iters = 0;
    long long solves = 0;     // step batches solved
};

namespace {

constexpr double CG_TOL = 1e-13;
constexpr int CG_MAX_ITER = 300;

// ---------------------------------------------------------------------------- printed entries

// Every printed entry with offset l >= 2 has the form
//     E(l) = sum_{s=-2..2} ( w p4 c3[s] (l + s)_+^{p3} + c4[s] (l + s)_+^{p4} ),  p4 = 4 - 2 rho, p3 = p4 - 1,
// high-order differences whose terms cancel to many digits for large l (E(l) ~ l^{p4 - 5}).  Expanding
// (l + s)^p = l^p sum_k binom(p, k) (s / l)^k and using binom(p4, k) = (p4 / k) binom(p3, k - 1),
//     E(l) = p4 l^{p4} sum_{k >= 1} binom(p3, k - 1) (m4_k / k + w m3_{k-1}) l^{-k},
// with the integer moments m_k = sum_s c[s] s^k (m4_0 = 0 for every entry).  The brackets of the
// orders that cancel are exact zeros (small integers), so nothing cancels in floating point.  The
// series converges for l >= 3 (|s / l| <= 2/3); offsets l <= 2 are summed directly.
double moment(const double c[5], int k) {
    double m = 0.0;
    for (int s = -2; s <= 2; ++s) {
        double q = 1.0;
        for (int e = 0; e < k; ++e) q *= (double)s;   // exact: |s| <= 2
        m += c[s + 2] * q;
    }
    return m;
}

double entry_series(int l, double p4, double w, const double c3[5], const double c4[5]) {
    const double p3 = p4 - 1.0;
    if (l <= 2) {
        double v = 0.0;
        for (int s = -2; s <= 2; ++s)
            if (l + s > 0) v += w * p4 * c3[s + 2] * pow((double)(l + s), p3) + c4[s + 2] * pow((double)(l + s), p4);
        return v;
    }
    const int K = l < 8 ? 220 : 80;
    double sum = 0.0, b = 1.0, lk = 1.0 / l;   // b = binom(p3, k - 1), lk = l^{-k}
    for (int k = 1; k <= K; ++k) {
        sum += b * (moment(c4, k) / k + w * moment(c3, k - 1)) * lk;
        b *= (p3 - (k - 1)) / (double)k;
        lk /= (double)l;
    }
    return p4 * pow((double)l, p4) * sum;
}

// a^{1,rho}_{k,k+l} (symmetric), a^{2,rho}_{k,k+l} (l >= 0) and a^{2,rho}_{p+m,p} (m >= 1), Sec. 2
double entry_a1(int l, double r) {
    if (l == 0) return pow(2.0, 6.0 - 2.0 * r) + 16.0 * r - 40.0;
    if (l == 1) return 2.0 * pow(3.0, 4.0 - 2.0 * r) + (2.0 * r - 6.0) * pow(2.0, 5.0 - 2.0 * r) - 16.0 * r + 34.0;
    const double c3[5] = {0.0, -1.0, 2.0, -1.0, 0.0}, c4[5] = {-2.0, 4.0, 0.0, -4.0, 2.0};
    return entry_series(l, 4.0 - 2.0 * r, 4.0, c3, c4);
}

double entry_a2_upper(int l, double r) {
    if (l <= 1) return 4.0 - pow(2.0, 4.0 - 2.0 * r) * r;
    const double c3[5] = {1.0, -1.0, -1.0, 1.0, 0.0}, c4[5] = {2.0, -6.0, 6.0, -2.0, 0.0};
    return entry_series(l, 4.0 - 2.0 * r, 1.0, c3, c4);
}

double entry_a2_lower(int m, double r) {
    const double c3[5] = {0.0, 1.0, -1.0, -1.0, 1.0}, c4[5] = {0.0, 2.0, -6.0, 6.0, -2.0};
    return entry_series(m, 4.0 - 2.0 * r, 1.0, c3, c4);
}

// A_2[i][l] of order n
double a2_at(const std::vector<double>& up, const std::vector<double>& lo, int i, int l) {
    return l >= i ? up[l - i] : lo[i - l];
}

void entries(int n, double rho, std::vector<double>& a1, std::vector<double>& up, std::vector<double>& lo) {
    a1.resize(n); up.resize(n); lo.assign(n, 0.0);
    for (int l = 0; l < n; ++l) {
        a1[l] = entry_a1(l, rho);
        up[l] = entry_a2_upper(l, rho);
        if (l >= 1) lo[l] = entry_a2_lower(l, rho);
    }
}

// ---------------------------------------------------------------------------- kernels

constexpr int BK = 16;

struct P1Args {
    // operand: V = V1 + sk V2 (stiffness input), Vm = V1 + sm V2 (mass input); V2 may be null
    const double* V1; const double* V2; long long vs; double sk, sm;
    const double* Mat;                    // Bx (x product) or By (y product)
    const double* T; long long ts;        // y product: the x product's output (or null: no x term)
    double* out; long long os;
    int Px, Py, nx, ny;
    double cxk, cyk;                      // c_x K_x and c_y K_y
    double mass_w;                        // h_x h_y / 12 times the mass coefficient (0: no mass term)
    double ksign, taum;                   // stiffness coefficient of slice b: ksign * taum * dt[n_b - 1]
    const double* dt; int n0, dn;         // n_b = n0 + b dn (dt null: coefficient ksign * taum)
    int load;                             // add F_{n_b}
    int rank; const double* time_w; const double* bxn; const double* byn; const double* Fd;
    const double* E; long long es;        // out = gE E + gO (...)  (E may be null)
    double gE, gO;
    double* partial;                      // per-CTA sums of out^2 (or null)
};

// MODE 0: T_b = [V | V_{j+1} | V_{j-1}] Bx  (Py x Px per slice)
// MODE 1: out_b = gE E_b + gO (mass_w M7(Vm) + k_b (c_x K_x T_b + c_y K_y By [V; V_{i+1}; V_{i-1}]) + F)
template <int TT, int MODE>
__global__ void __launch_bounds__(256) k_p1_gemm(P1Args a) {
    constexpr int MT = TT / 16;
    __shared__ double As[BK][TT + 1];
    __shared__ double Bs[BK][TT + 1];
    __shared__ double red[256];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * TT, j0 = blockIdx.y * TT;
    const long long b = blockIdx.z;
    const double* V1 = a.V1 + b * a.vs;
    const double* V2 = a.V2 ? a.V2 + b * a.vs : nullptr;
    const int P = MODE == 0 ? a.Px : a.Py;   // contraction extent per shift
    const int K = 3 * P;

    double acc[MT][MT];
#pragma unroll
    for (int u = 0; u < MT; ++u)
#pragma unroll
        for (int v = 0; v < MT; ++v) acc[u][v] = 0.0;

    for (int k0 = 0; k0 < K; k0 += BK) {
        const int s = k0 / P;                 // BK divides P: a K tile never straddles two shifts
        const int sh = s == 1 ? 1 : (s == 2 ? -1 : 0);
        for (int e = threadIdx.x; e < TT * BK; e += 256) {
            const int row = e / BK, kk = e % BK;
            const int j = j0 + row;
            double v;
            if (MODE == 0) {
                const int l = k0 + kk - s * P, jj = j + sh;
                v = 0.0;
                if (jj >= 0 && jj < a.ny && l < a.nx) {
                    const size_t o = (size_t)jj * a.Px + l;
                    v = V1[o];
                    if (V2) v += a.sk * V2[o];
                }
            } else {
                v = a.Mat[(size_t)j * K + k0 + kk];
            }
            As[kk][row] = v;
        }
        for (int e = threadIdx.x; e < TT * BK; e += 256) {
            const int kk = e / TT, col = e % TT;
            const int i = i0 + col;
            double v;
            if (MODE == 0) {
                v = a.Mat[(size_t)(k0 + kk) * a.Px + i];
            } else {
                const int l = k0 + kk - s * P, ii = i + sh;
                v = 0.0;
                if (ii >= 0 && ii < a.nx && l < a.ny) {
                    const size_t o = (size_t)l * a.Px + ii;
                    v = V1[o];
                    if (V2) v += a.sk * V2[o];
                }
            }
            Bs[kk][col] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double av[MT], bv[MT];
#pragma unroll
            for (int u = 0; u < MT; ++u) av[u] = As[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < MT; ++v) bv[v] = Bs[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < MT; ++u)
#pragma unroll
                for (int v = 0; v < MT; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }

    double sq = 0.0;
#pragma unroll
    for (int u = 0; u < MT; ++u) {
        const int j = j0 + ty + 16 * u;
#pragma unroll
        for (int v = 0; v < MT; ++v) {
            const int i = i0 + tx + 16 * v;
            const size_t o = (size_t)j * a.Px + i;
            if (MODE == 0) {
                a.out[b * a.os + o] = acc[u][v];
                continue;
            }
            double r = 0.0;
            if (i < a.nx && j < a.ny) {
                const int n = a.n0 + (int)b * a.dn;
                const double kb = a.ksign * a.taum * (a.dt ? a.dt[n - 1] : 1.0);
                double stiff = a.cyk * acc[u][v];
                if (a.T) stiff += a.cxk * a.T[b * a.ts + o];
                double val = kb * stiff;
                if (a.mass_w != 0.0) {
                    auto vm = [&](int jj, int ii) -> double {
                        if (jj < 0 || jj >= a.ny || ii < 0 || ii >= a.nx) return 0.0;
                        const size_t q = (size_t)jj * a.Px + ii;
                        return V2 ? V1[q] + a.sm * V2[q] : V1[q];
                    };
                    const double m7 = 6.0 * vm(j, i) + vm(j, i - 1) + vm(j, i + 1) + vm(j + 1, i) + vm(j + 1, i + 1) +
                                      vm(j - 1, i) + vm(j - 1, i - 1);
                    val += a.mass_w * m7;
                }
                if (a.load) {
                    double f = 0.0;
                    for (int q = 0; q < a.rank; ++q)
                        f += a.time_w[(size_t)(n - 1) * a.rank + q] * a.byn[(size_t)q * a.Py + j] *
                             a.bxn[(size_t)q * a.Px + i];
                    if (a.Fd) f += a.Fd[(size_t)(n - 1) * ((size_t)a.Px * a.Py) + o];
                    val += f;
                }
                r = a.gO * val;
                if (a.E) r += a.gE * a.E[b * a.es + o];
            }
            sq += r * r;
            a.out[b * a.os + o] = r;
        }
    }
    if (MODE == 1 && a.partial) {
        red[threadIdx.x] = sq;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            a.partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
    }
}

// out[b] = <X_b, Y_b> over n entries, fixed summation order (one block per slice)
__global__ void __launch_bounds__(256) k_p1_dot(const double* X, const double* Y, long long stride, size_t n,
                                                 double* out) {
    __shared__ double s[256];
    const long long b = blockIdx.x;
    const double* x = X + b * stride;
    const double* y = Y + b * stride;
    double a0 = 0.0, a1 = 0.0;
    size_t e = threadIdx.x;
    for (; e + 256 < n; e += 512) {
        a0 = fma(x[e], y[e], a0);
        a1 = fma(x[e + 256], y[e + 256], a1);
    }
    if (e < n) a0 = fma(x[e], y[e], a0);
    s[threadIdx.x] = a0 + a1;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = s[0];
}

// X += alpha P, R -= alpha Q with alpha_b = rz_b / pq_b (0 when pq_b = 0: a slice already solved)
__global__ void k_p1_update_xr(double* X, double* R, const double* P, const double* Q, long long stride, size_t n,
                               const double* rz, const double* pq) {
    const long long b = blockIdx.y;
    const double al = pq[b] != 0.0 ? rz[b] / pq[b] : 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t o = b * stride + e;
        X[o] = fma(al, P[o], X[o]);
        R[o] = fma(-al, Q[o], R[o]);
    }
}

// P = Z + beta P with beta_b = rzn_b / rz_b (0 when rz_b = 0)
__global__ void k_p1_update_p(double* P, const double* Z, long long stride, size_t n, const double* rzn,
                              const double* rz) {
    const long long b = blockIdx.y;
    const double be = rz[b] != 0.0 ? rzn[b] / rz[b] : 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t o = b * stride + e;
        P[o] = fma(be, P[o], Z[o]);
    }
}

// *out = max_b rr_b / rr0_b (0 for a zero right-hand side; +inf if a ratio is not finite)
__global__ void k_p1_max_ratio(const double* rr, const double* rr0, int batch, double* out) {
    __shared__ double s[256];
    double m = 0.0;
    for (int b = threadIdx.x; b < batch; b += 256) {
        double q = rr0[b] > 0.0 ? rr[b] / rr0[b] : 0.0;
        if (!(q == q) || isinf(q)) q = INFINITY;
        m = fmax(m, q);
    }
    s[threadIdx.x] = m;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// ref_b = max(ref_b, other_b): the reference of the relative stopping test
__global__ void k_p1_max_into(double* ref, const double* other, int nb) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        ref[b] = fmax(ref[b], other[b]);
}

// X_b = guess_b (- g_b): the starting iterate of CG from an estimate of Phi(u) + g
__global__ void k_p1_init_x(double* X, long long xs, const double* guess, long long gs, const double* g, long long ggs,
                            size_t n) {
    const long long b = blockIdx.y;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double v = guess[b * gs + e];
        if (g) v -= g[b * ggs + e];
        X[b * xs + e] = v;
    }
}

// dst_b = X_b (+ g_b) (- u_b), with per-CTA sums of dst^2
__global__ void __launch_bounds__(256) k_p1_finish(const double* X, long long xs, const double* g, long long gs,
                                                   const double* ut, long long us, double* dst, long long ds, size_t n,
                                                   double* partial) {
    __shared__ double red[256];
    const long long b = blockIdx.y;
    double sq = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double v = X[b * xs + e];
        if (g) v += g[b * gs + e];
        if (ut) v -= ut[b * us + e];
        dst[b * ds + e] = v;
        sq += v * v;
    }
    if (partial) {
        red[threadIdx.x] = sq;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(size_t)b * gridDim.x + blockIdx.x] = red[0];
    }
}

int tile_for(int Px, int Py, long long batch) {
    int T = 64;
    while (T > 16 && (T > Px || T > Py || (long long)(Px / T) * (Py / T) * batch < 2 * 152)) T /= 2;
    return T;
}

template <int MODE>
void launch_gemm(sfde_ctx* c, int T, const P1Args& a, int batch) {
    const dim3 grid((unsigned)(a.Px / T), (unsigned)(a.Py / T), (unsigned)batch);
    const int slot = sfde_prof_begin(c);
    if (T == 64) k_p1_gemm<64, MODE><<<grid, 256, 0, c->stream>>>(a);
    else if (T == 32) k_p1_gemm<32, MODE><<<grid, 256, 0, c->stream>>>(a);
    else k_p1_gemm<16, MODE><<<grid, 256, 0, c->stream>>>(a);
    const double nx = c->x.n, ny = c->y.n;
    const double flops = 2.0 * batch * nx * ny * 3.0 * (MODE == 0 ? nx : ny);
    sfde_prof_end(c, slot, 6, flops, 8.0 * batch * (2.0 * nx * ny) + 8.0 * 3.0 * (MODE == 0 ? nx * nx : ny * ny));
    sfde_count_launch(c);
}

// Operator application on `batch` padded slices: see P1Args.  Partial sums (if asked for) are
// written per CTA of the second product: (Px/T)(Py/T) per slice; returns their count in *npart.
struct Apply {
    const double* V1 = nullptr; const double* V2 = nullptr; long long vs = 0; double sk = 0, sm = 0;
    double mass = 1.0;                  // coefficient of M_h
    double ksign = 1.0, taum = 0.5;     // stiffness coefficient ksign * taum * dt[n_b - 1]
    const double* dt = nullptr; int n0 = 1, dn = 1;
    bool load = false;
    const double* E = nullptr; long long es = 0; double gE = 0, gO = 1;
    double* out = nullptr; long long os = 0;
    double* partial = nullptr;
};

sfde_status p1_apply(sfde_ctx* c, const Apply& A, int batch, double* T, int* npart) {
    SfdeP1& p = *c->p1;
    const int Px = c->x.P, Py = c->y.P;
    const long long P2 = (long long)c->P2();
    const int TT = tile_for(Px, Py, std::min(batch, 65535));
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(batch - b0, 65535);
        P1Args a{};
        a.V1 = A.V1 + (long long)b0 * A.vs; a.V2 = A.V2 ? A.V2 + (long long)b0 * A.vs : nullptr; a.vs = A.vs;
        a.sk = A.sk; a.sm = A.sm;
        a.Px = Px; a.Py = Py; a.nx = c->x.n; a.ny = c->y.n;
        // x product into T (the stiffness input V1 + sk V2)
        a.Mat = p.Bx; a.out = T; a.os = P2;
        launch_gemm<0>(c, TT, a, nb);
        // y product, epilogue
        a.Mat = p.By; a.T = T; a.ts = P2;
        a.out = A.out + (long long)b0 * A.os; a.os = A.os;
        a.cxk = p.cx * c->kx; a.cyk = p.cy * c->ky;
        a.mass_w = A.mass * p.hx * p.hy / 12.0;
        a.ksign = A.ksign; a.taum = A.taum; a.dt = A.dt; a.n0 = A.n0 + b0 * A.dn; a.dn = A.dn;
        a.load = A.load ? 1 : 0; a.rank = c->rank; a.time_w = c->time_w; a.bxn = c->bxn; a.byn = c->byn; a.Fd = c->Fd;
        a.E = A.E ? A.E + (long long)b0 * A.es : nullptr; a.es = A.es; a.gE = A.gE; a.gO = A.gO;
        a.partial = A.partial ? A.partial + (size_t)b0 * (Px / TT) * (Py / TT) : nullptr;
        launch_gemm<1>(c, TT, a, nb);
    }
    if (npart) *npart = batch * (Px / TT) * (Py / TT);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

sfde_status p1_ensure(sfde_ctx* c, size_t slices) {
    SfdeP1& p = *c->p1;
    if (p.ws_slices >= slices) return SFDE_OK;
    cudaFree(p.ws); cudaFree(p.dots);
    p.ws = p.dots = nullptr;
    p.ws_slices = 0;
    SFDE_CUDA(cudaMalloc(&p.ws, sizeof(double) * 7 * slices * c->P2()));
    SFDE_CUDA(cudaMalloc(&p.dots, sizeof(double) * 6 * slices));
    p.ws_slices = slices;
    return SFDE_OK;
}

void launch_dot(sfde_ctx* c, const double* X, const double* Y, int nb, double* out) {
    k_p1_dot<<<nb, 256, 0, c->stream>>>(X, Y, (long long)c->P2(), c->P2(), out);
    sfde_count_launch(c);
}

dim3 vec_grid(sfde_ctx* c, int nb) {
    const unsigned per = (unsigned)std::min<size_t>((c->P2() + 255) / 256, std::max(1, 1216 / std::max(1, nb)));
    return dim3(std::max(1u, per), (unsigned)nb);
}

// X_b = S_b^{-1} R_b for nb slices (contiguous in the workspace), S_b = M_h + taum dt[n_b-1] K, from
// X = guess - g when an estimate is given, else from X = 0; converged when every slice's residual is
// below 1e-13 of the larger of its ||R|| and its initial residual
sfde_status p1_pcg(sfde_ctx* c, int nb, const double* dt, int n0, int dn, double taum, int solve_scheme,
                   const double* guess, long long guess_stride, const double* g, long long g_stride) {
    SfdeP1& p = *c->p1;
    const long long P2 = (long long)c->P2();
    const size_t n = c->P2();
    double* R = p.ws;
    double* X = R + (size_t)nb * P2;
    double* r = X + (size_t)nb * P2;
    double* z = r + (size_t)nb * P2;
    double* pv = z + (size_t)nb * P2;
    double* q = pv + (size_t)nb * P2;
    double* T = q + (size_t)nb * P2;
    double* rr0 = p.dots;
    double* rz = rr0 + nb;
    double* rzn = rz + nb;
    double* pq = rzn + nb;
    double* rr = pq + nb;
    double* mx = rr + nb;
    auto precond = [&](const double* in, double* outp) {
        return sfde_fdm_solve_fp64(c, in, P2, outp, P2, nb, dt, n0, dn, solve_scheme);
    };
    auto apply_S = [&](const double* in, double* outp, const double* E, double gE, double gO) {
        Apply A;
        A.V1 = in; A.vs = P2; A.mass = 1.0; A.ksign = 1.0; A.taum = taum; A.dt = dt; A.n0 = n0; A.dn = dn;
        A.E = E; A.es = P2; A.gE = gE; A.gO = gO; A.out = outp; A.os = P2;
        return p1_apply(c, A, nb, T, nullptr);
    };
    const dim3 vg = vec_grid(c, nb);
    // x0 = guess - g (or 0), r = R - S x0, z = P^{-1} r, p = z
    if (guess) {
        k_p1_init_x<<<vg, 256, 0, c->stream>>>(X, P2, guess, guess_stride, g, g_stride, n);
        sfde_count_launch(c);
        SFDE_TRY(apply_S(X, r, R, 1.0, -1.0));
    } else {
        SFDE_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * n * nb, c->stream));
        SFDE_CUDA(cudaMemcpyAsync(r, R, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, c->stream));
    }
    // the stopping test is relative to the larger of ||R|| and the initial residual: a zero right-hand
    // side (a zeroed coarse iterate) with a nonzero starting value must still be solved
    launch_dot(c, R, R, nb, rr0);
    if (guess) {
        launch_dot(c, r, r, nb, rr);
        k_p1_max_into<<<(nb + 255) / 256, 256, 0, c->stream>>>(rr0, rr, nb);
        sfde_count_launch(c);
    }
    SFDE_TRY(precond(r, z));
    SFDE_CUDA(cudaMemcpyAsync(pv, z, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, c->stream));
    launch_dot(c, r, z, nb, rz);
    int it = 0;
    bool done = false;
    const double tol2 = CG_TOL * CG_TOL;
    for (it = 1; it <= CG_MAX_ITER; ++it) {
        SFDE_TRY(apply_S(pv, q, nullptr, 0.0, 1.0));
        launch_dot(c, pv, q, nb, pq);
        k_p1_update_xr<<<vg, 256, 0, c->stream>>>(X, r, pv, q, P2, n, rz, pq);
        sfde_count_launch(c);
        launch_dot(c, r, r, nb, rr);
        k_p1_max_ratio<<<1, 256, 0, c->stream>>>(rr, rr0, nb, mx);
        sfde_count_launch(c);
        SFDE_CUDA(cudaMemcpyAsync(p.hmax, mx, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SFDE_CUDA(cudaStreamSynchronize(c->stream));
        const double ratio = *p.hmax;
        if (!(ratio <= 1e300)) break;            // not finite: report non-convergence
        if (ratio <= tol2) { done = true; break; }
        SFDE_TRY(precond(r, z));
        launch_dot(c, r, z, nb, rzn);
        k_p1_update_p<<<vg, 256, 0, c->stream>>>(pv, z, P2, n, rzn, rz);
        sfde_count_launch(c);
        std::swap(rz, rzn);
    }
    p.last_iters = it;
    p.total_iters += it;
    p.solves += 1;
    SFDE_CUDA(cudaGetLastError());
    return done ? SFDE_OK : SFDE_ENOCONV;
}

}  // namespace

// ---------------------------------------------------------------------------- setup / teardown

sfde_status sfde_p1_setup(sfde_ctx* c) {
    c->p1 = new (std::nothrow) SfdeP1();
    if (!c->p1) return SFDE_ENOMEM;
    SfdeP1& p = *c->p1;
    const int nx = c->x.n, ny = c->y.n, Px = c->x.P, Py = c->y.P;
    const double bx = c->x.rho, gy = c->y.rho;
    p.hx = c->x.h; p.hy = c->y.h;
    p.cx = pow(p.hx, 1.0 - 2.0 * bx) * p.hy / (2.0 * cos(bx * M_PI) * tgamma(5.0 - 2.0 * bx));
    p.cy = p.hx * pow(p.hy, 1.0 - 2.0 * gy) / (2.0 * cos(gy * M_PI) * tgamma(5.0 - 2.0 * gy));
    std::vector<double> a1, up, lo;
    // Bx rows k = s Px + l: s = 0 A_1[l][i], s = 1 A_2^T[l][i] = A_2[i][l], s = 2 A_2[l][i]
    entries(nx, bx, a1, up, lo);
    std::vector<double> hB((size_t)3 * Px * Px, 0.0);
    for (int l = 0; l < nx; ++l)
        for (int i = 0; i < nx; ++i) {
            hB[(size_t)l * Px + i] = a1[std::abs(l - i)];
            hB[((size_t)Px + l) * Px + i] = a2_at(up, lo, i, l);
            hB[((size_t)2 * Px + l) * Px + i] = a2_at(up, lo, l, i);
        }
    SFDE_CUDA(cudaMalloc(&p.Bx, sizeof(double) * hB.size()));
    SFDE_CUDA(cudaMemcpy(p.Bx, hB.data(), sizeof(double) * hB.size(), cudaMemcpyHostToDevice));
    // By[j][s Py + l]: s = 0 A_1[j][l], s = 1 A_2[j][l], s = 2 A_2^T[j][l] = A_2[l][j]
    entries(ny, gy, a1, up, lo);
    std::vector<double> hC((size_t)3 * Py * Py, 0.0);
    for (int j = 0; j < ny; ++j)
        for (int l = 0; l < ny; ++l) {
            hC[(size_t)j * 3 * Py + l] = a1[std::abs(j - l)];
            hC[(size_t)j * 3 * Py + Py + l] = a2_at(up, lo, j, l);
            hC[(size_t)j * 3 * Py + 2 * Py + l] = a2_at(up, lo, l, j);
        }
    SFDE_CUDA(cudaMalloc(&p.By, sizeof(double) * hC.size()));
    SFDE_CUDA(cudaMemcpy(p.By, hC.data(), sizeof(double) * hC.size(), cudaMemcpyHostToDevice));
    SFDE_CUDA(cudaMallocHost(&p.hmax, sizeof(double)));
    return SFDE_OK;
}

void sfde_p1_free(sfde_ctx* c) {
    if (!c || !c->p1) return;
    SfdeP1& p = *c->p1;
    cudaFree(p.Bx); cudaFree(p.By); cudaFree(p.ws); cudaFree(p.dots);
    if (p.hmax) cudaFreeHost(p.hmax);
    delete c->p1;
    c->p1 = nullptr;
}

// ---------------------------------------------------------------------------- step, residuals

// The fine or coarse step of StepBatch with the P1 matrices: R = B U (+ F_n) for CN (M_h U for the
// backward-Euler coarse propagator), X = S^{-1} R by PCG, dst = X (+ g) (- u_target) with per-CTA
// sums of squares in sb.norm_partial.
sfde_status sfde_step_p1(sfde_ctx* c, const StepBatch& sb, int* n_partials) {
    const long long P2 = (long long)c->P2();
    // chunks of at most the step workspace's slices (the preconditioner's scratch) and 4096
    const size_t chunk = std::max<size_t>(1, std::min<size_t>({c->ws_slices ? c->ws_slices : 1, (size_t)4096,
                                                              (size_t)sb.batch}));
    if (c->ws_slices < chunk) {
        // a norm buffer handed in is the context's own, which growing the workspace would replace
        if (sb.norm_partial) return SFDE_EINVAL;
        SFDE_TRY(sfde_ensure_workspace(c, chunk));
    }
    SFDE_TRY(p1_ensure(c, chunk));
    const bool cn = sb.scheme == SCHEME_CN;
    const double taum = cn ? 0.5 : 1.0;
    int total = 0;
    sfde_status rc = SFDE_OK;
    for (int b0 = 0; b0 < sb.batch; b0 += (int)chunk) {
        const int nb = std::min<int>(sb.batch - b0, (int)chunk);
        double* R = c->p1->ws;
        double* T = R + (size_t)6 * nb * P2;    // the last workspace buffer (p1_pcg's layout)
        const int n0 = sb.n0 + b0 * sb.dn;
        Apply A;
        A.V1 = sb.src + (long long)b0 * sb.src_stride; A.vs = sb.src_stride;
        A.mass = 1.0; A.ksign = cn ? -1.0 : 0.0; A.taum = taum; A.dt = sb.dt; A.n0 = n0; A.dn = sb.dn;
        A.load = sb.level0 && (c->rank > 0 || c->Fd);
        A.out = R; A.os = P2;
        SFDE_TRY(p1_apply(c, A, nb, T, nullptr));
        sfde_status st = p1_pcg(c, nb, sb.dt, n0, sb.dn, taum, cn ? SCHEME_SOLVE : SCHEME_SOLVE_BE,
                                sb.guess ? sb.guess + (long long)b0 * sb.guess_stride : nullptr, sb.guess_stride,
                                sb.g ? sb.g + (long long)b0 * sb.g_stride : nullptr, sb.g_stride);
        if (st != SFDE_OK && st != SFDE_ENOCONV) return st;
        if (st == SFDE_ENOCONV) rc = SFDE_ENOCONV;
        const double* X = c->p1->ws + (size_t)nb * P2;     // the CG iterate
        const dim3 vg = vec_grid(c, nb);
        if (sb.norm_partial && (size_t)total + (size_t)vg.x * nb > c->partial_cap) return SFDE_EINVAL;
        k_p1_finish<<<vg, 256, 0, c->stream>>>(X, P2, sb.g ? sb.g + (long long)b0 * sb.g_stride : nullptr, sb.g_stride,
                                              sb.utgt ? sb.utgt + (long long)b0 * sb.utgt_stride : nullptr,
                                              sb.utgt_stride, sb.dst + (long long)b0 * sb.dst_stride, sb.dst_stride,
                                              c->P2(), sb.norm_partial ? sb.norm_partial + total : nullptr);
        sfde_count_launch(c);
        total += (int)vg.x * nb;
    }
    SFDE_CUDA(cudaGetLastError());
    if (n_partials) *n_partials = total;
    return rc;
}

// sum over n = 1..N_t of ||rho_n||^2, rho_n = F_n + M_h (U_{n-1} - U_n) - tau_n K (U_{n-1} + U_n)
sfde_status sfde_residual_norm2_p1(sfde_ctx* c, const double* U, double* norm2) {
    const long long P2 = (long long)c->P2();
    SFDE_TRY(sfde_ensure_workspace(c, 1));
    const size_t chunk = std::max<size_t>(1, c->ws_slices);
    SFDE_TRY(p1_ensure(c, chunk));
    double acc = 0.0;
    for (int n0 = 1; n0 <= c->nt; n0 += (int)chunk) {
        const int nb = std::min<int>(c->nt - n0 + 1, (int)chunk);
        Apply A;
        A.V1 = U + (size_t)(n0 - 1) * P2; A.V2 = U + (size_t)n0 * P2; A.vs = P2; A.sk = 1.0; A.sm = -1.0;
        A.mass = 1.0; A.ksign = -1.0; A.taum = 0.5; A.dt = c->dt0; A.n0 = n0; A.dn = 1; A.load = true;
        A.out = c->p1->ws; A.os = P2; A.partial = c->partial;
        int np = 0;
        if ((size_t)nb * (c->x.P / 16) * (c->y.P / 16) > c->partial_cap) return SFDE_EINVAL;
        SFDE_TRY(p1_apply(c, A, nb, c->p1->ws + (size_t)nb * P2, &np));
        double r2 = 0.0;
        SFDE_TRY(sfde_reduce_partials(c, np, &r2));
        acc += r2;
    }
    *norm2 = acc;
    return SFDE_OK;
}

// sum over b < count of ||S_{n0 + b dn} R_b||^2 with the P1 matrices
sfde_status sfde_apply_S_norm2_p1(sfde_ctx* c, const double* R, long long r_stride, int count, int n0, int dn,
                                  double* norm2) {
    const long long P2 = (long long)c->P2();
    const size_t chunk = std::max<size_t>(1, c->ws_slices);
    SFDE_TRY(p1_ensure(c, chunk));
    double acc = 0.0;
    for (int b0 = 0; b0 < count; b0 += (int)chunk) {
        const int nb = std::min<int>(count - b0, (int)chunk);
        Apply A;
        A.V1 = R + (long long)b0 * r_stride; A.vs = r_stride;
        A.mass = 1.0; A.ksign = 1.0; A.taum = 0.5; A.dt = c->dt0; A.n0 = n0 + b0 * dn; A.dn = dn;
        A.out = c->p1->ws; A.os = P2; A.partial = c->partial;
        int np = 0;
        if ((size_t)nb * (c->x.P / 16) * (c->y.P / 16) > c->partial_cap) return SFDE_EINVAL;
        SFDE_TRY(p1_apply(c, A, nb, c->p1->ws + (size_t)nb * P2, &np));
        double r2 = 0.0;
        SFDE_TRY(sfde_reduce_partials(c, np, &r2));
        acc += r2;
    }
    *norm2 = acc;
    return SFDE_OK;
}

// ---------------------------------------------------------------------------- C ABI hooks

extern "C" sfde_status sfde_debug_p1_entries(int n, double rho, double* a1, double* a2_upper, double* a2_lower) {
    if (n < 1 || !(rho > 0.5 && rho <= 1.0) || !a1 || !a2_upper || !a2_lower) return SFDE_EINVAL;
    return sfde_no_throw([&] {
        std::vector<double> v1, up, lo;
        entries(n, rho, v1, up, lo);
        memcpy(a1, v1.data(), sizeof(double) * n);
        memcpy(a2_upper, up.data(), sizeof(double) * n);
        memcpy(a2_lower, lo.data(), sizeof(double) * n);
        return SFDE_OK;
    });
}

// out_b = (M_h + s_b K) U_b with s_b = tau_{n0 + b dn} (the S of Eq. (2.4)) for `batch` unpadded slices on
// the device (verification of the operator against its printed form)
extern "C" sfde_status sfde_debug_p1_apply_S(sfde_ctx* c, const double* U, int batch, int n0, int dn, double* out) {
    if (!c || !c->p1 || !U || !out || batch < 1 || n0 < 1 || n0 + (long long)(batch - 1) * dn > c->nt ||
        n0 + (long long)(batch - 1) * dn < 1)
        return SFDE_EINVAL;
    return sfde_no_throw([&]() -> sfde_status {
        const long long P2 = (long long)c->P2();
        SFDE_TRY(p1_ensure(c, (size_t)batch));
        double* in = c->p1->ws;
        double* o = in + (size_t)batch * P2;
        double* T = o + (size_t)batch * P2;
        sfde_launch_pad(U, in, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
        Apply A;
        A.V1 = in; A.vs = P2; A.mass = 1.0; A.ksign = 1.0; A.taum = 0.5; A.dt = c->dt0; A.n0 = n0; A.dn = dn;
        A.out = o; A.os = P2;
        SFDE_TRY(p1_apply(c, A, batch, T, nullptr));
        sfde_launch_unpad(o, out, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
        SFDE_CUDA(cudaGetLastError());
        SFDE_CUDA(cudaStreamSynchronize(c->stream));
        return SFDE_OK;
    });
}

// CG iterations of the last step batch, and the total over all step batches and their count
extern "C" sfde_status sfde_debug_p1_cg_stats(sfde_ctx* c, int* last, long long* total, long long* solves) {
    if (!c || !c->p1) return SFDE_EINVAL;
    if (last) *last = c->p1->last_iters;
    if (total) *total = c->p1->total_iters;
    if (solves) *solves = c->p1->solves;
    return SFDE_OK;
}
