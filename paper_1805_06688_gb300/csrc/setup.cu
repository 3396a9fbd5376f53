// Setup of one spatial direction on the device, all in FP64 (Sec. 2):
//   * Toeplitz coefficients of the 1-D linear-element Riesz stiffness,
//   * the dense padded stiffness A,
//   * generalised eigenpairs A V = M V diag(lambda), V^T M V = I, through M = L L^T
//     (tridiagonal Cholesky), C = L^{-1} A L^{-T} and parallel cyclic Jacobi rotations,
//   * W = M V and the transposed operand copies used by the step GEMMs.
// Also small layout kernels (padding, strided axpy, the SplitMix64 initial guess).
#include <math.h>
#include <stdio.h>

#include "sfde_internal.cuh"

namespace {

// ----------------------------------------------------------------------------------------
// Toeplitz coefficients.  With p = 3 - 2 rho and c = (1,-4,6,-4,1),
//   g(k) = sum_{s=-2..2} c_s (k+s)_+^p,   a_k = pref * (g(k) + g(-k)),
//   pref = h^{1-2rho} / (2 cos(rho pi) Gamma(4 - 2 rho))   (from the element integrals, Sec. 2).
// g(-k) vanishes for k >= 2 and g(-1) = 1.  For k >= 3 the fourth difference is summed as the
// binomial series  g(k) = k^p sum_{j = 4,6,8,..} binom(p, j) 2 (2^j - 4) k^{-j}, whose terms are
// all positive for 1 < p < 2 (no cancellation), instead of differencing k^p directly.
__global__ void k_toeplitz_coeffs(double* a, int n, double p, double pref) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double g;
    if (k == 0) {
        g = 2.0 * (pow(2.0, p) - 4.0);
    } else if (k == 1) {
        g = pow(3.0, p) - 4.0 * pow(2.0, p) + 7.0;
    } else if (k == 2) {
        g = -4.0 + 6.0 * pow(2.0, p) - 4.0 * pow(3.0, p) + pow(4.0, p);
    } else {
        const double x = 1.0 / (double)k;
        const double x2 = x * x;
        // binom(p, j) for j = 0..3 then step by two
        double b = p * (p - 1.0) * (p - 2.0) * (p - 3.0) / 24.0;  // binom(p,4)
        double xj = x2 * x2;                                        // k^-4
        double two_j = 16.0;                                        // 2^j
        double sum = 0.0;
        for (int j = 4; j < 400; j += 2) {
            double term = b * 2.0 * (two_j - 4.0) * xj;
            sum += term;
            if (fabs(term) <= 1e-18 * fabs(sum)) break;
            // advance binom(p, j) -> binom(p, j+2)
            b *= (p - j) * (p - j - 1.0) / ((j + 1.0) * (j + 2.0));
            xj *= x2;
            two_j *= 4.0;
        }
        g = pow((double)k, p) * sum;
    }
    a[k] = pref * g;
}

__global__ void k_toeplitz_dense(const double* a, double* A, int n, int P) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= P) return;
    A[(size_t)i * P + j] = (i < n && j < n) ? a[abs(i - j)] : 0.0;
}

// Tridiagonal Cholesky of M = (h/6) tridiag(1,4,1): L has diagonal l[i] and subdiagonal e[i] = L[i+1][i].
__global__ void k_mass_cholesky(double* l, double* e, int n, double h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double d = 4.0 * h / 6.0, o = h / 6.0;
    double prev = sqrt(d);
    l[0] = prev;
    for (int i = 1; i < n; ++i) {
        double ei = o / prev;
        e[i - 1] = ei;
        prev = sqrt(d - ei * ei);
        l[i] = prev;
    }
}

// Y = L^{-1} X, one thread per column (X, Y: n x n, leading dimension ld).
__global__ void k_forward_subst_cols(const double* X, double* Y, int n, int ld, const double* l,
                                     const double* e) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double y = X[c] / l[0];
    Y[c] = y;
    for (int i = 1; i < n; ++i) {
        y = (X[(size_t)i * ld + c] - e[i - 1] * y) / l[i];
        Y[(size_t)i * ld + c] = y;
    }
}

// C[:, r] = L^{-1} (row r of Y)^T, one thread per r: C = L^{-1} Y^T.
__global__ void k_forward_subst_rows_T(const double* Y, double* C, int n, int ld, const double* l,
                                       const double* e) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double z = Y[(size_t)r * ld] / l[0];
    C[r] = z;
    for (int i = 1; i < n; ++i) {
        z = (Y[(size_t)r * ld + i] - e[i - 1] * z) / l[i];
        C[(size_t)i * ld + r] = z;
    }
}

__global__ void k_symmetrize(double* C, int ne, int n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= ne) return;
    if (i >= n || j >= n) {
        C[(size_t)i * ne + j] = 0.0;
        return;
    }
    if (j <= i) return;
    double v = 0.5 * (C[(size_t)i * ne + j] + C[(size_t)j * ne + i]);
    C[(size_t)i * ne + j] = v;
    C[(size_t)j * ne + i] = v;
}

__global__ void k_identity(double* Q, int ne) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= ne) return;
    Q[(size_t)i * ne + j] = (i == j) ? 1.0 : 0.0;
}

// Round-robin ("circle") pairing of ne indices: over rounds 0..ne-2 every unordered pair
// appears once and every index appears once per round.
__device__ __forceinline__ int rr_player(int pos, int round, int ne) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (ne - 1)) + 1;
}

struct Rot { int p, q; double c, s; };

// Jacobi rotation for each pair of this round: J = [[c, s], [-s, c]] on (p, q) with J^T C J
// diagonal on that 2x2 block (symmetric Schur decomposition of the block).
__global__ void k_jacobi_rotations(const double* C, int ne, int round, Rot* rot) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne / 2) return;
    int p = rr_player(k, round, ne), q = rr_player(ne - 1 - k, round, ne);
    double app = C[(size_t)p * ne + p], aqq = C[(size_t)q * ne + q], apq = C[(size_t)p * ne + q];
    double c = 1.0, s = 0.0;
    if (apq != 0.0) {
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
    }
    rot[k] = Rot{p, q, c, s};
}

// C <- J^T C J on every 2x2 block (pair a rows, pair b columns); the blocks are disjoint.
__global__ void k_jacobi_apply(double* C, int ne, const Rot* rot) {
    int half = ne / 2;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    int a = blockIdx.y;
    if (b >= half) return;
    Rot ra = rot[a], rb = rot[b];
    size_t pp = (size_t)ra.p * ne + rb.p, pq = (size_t)ra.p * ne + rb.q;
    size_t qp = (size_t)ra.q * ne + rb.p, qq = (size_t)ra.q * ne + rb.q;
    double w = C[pp], x = C[pq], y = C[qp], z = C[qq];
    // columns (pair b)
    double w1 = rb.c * w - rb.s * x, x1 = rb.s * w + rb.c * x;
    double y1 = rb.c * y - rb.s * z, z1 = rb.s * y + rb.c * z;
    // rows (pair a)
    double w2 = ra.c * w1 - ra.s * y1, y2 = ra.s * w1 + ra.c * y1;
    double x2 = ra.c * x1 - ra.s * z1, z2 = ra.s * x1 + ra.c * z1;
    if (a == b) { x2 = 0.0; y2 = 0.0; }
    C[pp] = w2; C[pq] = x2; C[qp] = y2; C[qq] = z2;
}

__global__ void k_jacobi_apply_Q(double* Q, int ne, const Rot* rot) {
    int half = ne / 2;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (b >= half) return;
    Rot rb = rot[b];
    size_t ip = (size_t)i * ne + rb.p, iq = (size_t)i * ne + rb.q;
    double u = Q[ip], v = Q[iq];
    Q[ip] = rb.c * u - rb.s * v;
    Q[iq] = rb.s * u + rb.c * v;
}

// The whole Jacobi iteration in one CTA for small even orders (ne <= 64): C and Q held in shared
// memory, the same rotations applied in the same rounds as k_jacobi_rotations / k_jacobi_apply /
// k_jacobi_apply_Q, sweeps until the off-diagonal mass falls to the rounding floor (at most
// max_sweeps).  Leading dimension ne in global and shared memory.
constexpr int JACOBI_SMEM_MAX = 64;
__global__ void __launch_bounds__(256) k_jacobi_small(double* Cg, double* Qg, int ne, int max_sweeps) {
    extern __shared__ double sm[];
    double* C = sm;
    double* Q = sm + ne * ne;
    __shared__ Rot rot[JACOBI_SMEM_MAX / 2];
    __shared__ double so[256], sd[256];
    __shared__ int done;
    const int half = ne / 2;
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) { C[e] = Cg[e]; Q[e] = Qg[e]; }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < ne - 1; ++round) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                const int p = rr_player(k, round, ne), q = rr_player(ne - 1 - k, round, ne);
                const double app = C[p * ne + p], aqq = C[q * ne + q], apq = C[p * ne + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (aqq - app) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                rot[k] = Rot{p, q, c, s};
            }
            __syncthreads();
            for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
                const int a = e / half, b = e % half;
                const Rot ra = rot[a], rb = rot[b];
                const int pp = ra.p * ne + rb.p, pq = ra.p * ne + rb.q, qp = ra.q * ne + rb.p, qq = ra.q * ne + rb.q;
                const double w = C[pp], x = C[pq], y = C[qp], z = C[qq];
                const double w1 = rb.c * w - rb.s * x, x1 = rb.s * w + rb.c * x;
                const double y1 = rb.c * y - rb.s * z, z1 = rb.s * y + rb.c * z;
                const double w2 = ra.c * w1 - ra.s * y1, y2 = ra.s * w1 + ra.c * y1;
                double x2 = ra.c * x1 - ra.s * z1, z2 = ra.s * x1 + ra.c * z1;
                double y2b = y2;
                if (a == b) { x2 = 0.0; y2b = 0.0; }
                C[pp] = w2; C[pq] = x2; C[qp] = y2b; C[qq] = z2;
            }
            for (int e = threadIdx.x; e < ne * half; e += blockDim.x) {
                const int i = e / half, b = e % half;
                const Rot rb = rot[b];
                const double u = Q[i * ne + rb.p], v = Q[i * ne + rb.q];
                Q[i * ne + rb.p] = rb.c * u - rb.s * v;
                Q[i * ne + rb.q] = rb.s * u + rb.c * v;
            }
            __syncthreads();
        }
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
            const double v = C[e];
            if (e / ne == e % ne) dg += v * v; else off += v * v;
        }
        so[threadIdx.x] = off;
        sd[threadIdx.x] = dg;
        __syncthreads();
        for (int k = blockDim.x / 2; k > 0; k >>= 1) {
            if ((int)threadIdx.x < k) { so[threadIdx.x] += so[threadIdx.x + k]; sd[threadIdx.x] += sd[threadIdx.x + k]; }
            __syncthreads();
        }
        if (threadIdx.x == 0) done = so[0] <= 1e-30 * (double)ne * sd[0];
        __syncthreads();
        if (done) break;
    }
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) { Cg[e] = C[e]; Qg[e] = Q[e]; }
}

__global__ void k_offdiag_norm(const double* C, int ne, double* out /* [off, diag] */) {
    __shared__ double so[256], sd[256];
    double off = 0.0, dg = 0.0;
    size_t total = (size_t)ne * ne;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        size_t i = idx / ne, j = idx % ne;
        double v = C[idx];
        if (i == j) dg += v * v; else off += v * v;
    }
    so[threadIdx.x] = off;
    sd[threadIdx.x] = dg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { so[threadIdx.x] += so[threadIdx.x + s]; sd[threadIdx.x] += sd[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { atomicAdd(&out[0], so[0]); atomicAdd(&out[1], sd[0]); }
}

// V = L^{-T} Q restricted to the first n rows/columns, written zero padded (P x P); lambda = diag C.
__global__ void k_back_subst_eigvec(const double* Q, const double* C, int ne, int n, int P,
                                    const double* l, const double* e, double* V, double* lam) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    if (k >= n) {
        for (int i = 0; i < P; ++i) V[(size_t)i * P + k] = 0.0;
        lam[k] = 1.0;
        return;
    }
    double v = Q[(size_t)(n - 1) * ne + k] / l[n - 1];
    V[(size_t)(n - 1) * P + k] = v;
    for (int i = n - 2; i >= 0; --i) {
        v = (Q[(size_t)i * ne + k] - e[i] * v) / l[i];
        V[(size_t)i * P + k] = v;
    }
    for (int i = n; i < P; ++i) V[(size_t)i * P + k] = 0.0;
    lam[k] = C[(size_t)k * ne + k];
}

// W = M V with M = (h/6) tridiag(1,4,1) on the first n rows.
__global__ void k_mass_apply_cols(const double* V, double* W, int n, int P, double h) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (k >= P) return;
    double w = 0.0;
    if (i < n) {
        double c = V[(size_t)i * P + k];
        double up = i > 0 ? V[(size_t)(i - 1) * P + k] : 0.0;
        double dn = i + 1 < n ? V[(size_t)(i + 1) * P + k] : 0.0;
        w = (h / 6.0) * (up + 4.0 * c + dn);
    }
    W[(size_t)i * P + k] = w;
}

__global__ void k_transpose(const double* X, double* Y, int P) {
    __shared__ double tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y)
        tile[r][threadIdx.x] = X[(size_t)(by + r) * P + bx + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y)
        Y[(size_t)(bx + r) * P + by + threadIdx.x] = tile[threadIdx.x][r];
}

// p[r][k] = sum_i b[r][i] V[i][k]: modal coefficients of the separable load factors.
__global__ void k_project_factor(const double* b, const double* V, double* p, int rank, int n, int P) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (k >= P || r >= rank) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += b[(size_t)r * n + i] * V[(size_t)i * P + k];
    p[(size_t)r * P + k] = s;
}

__global__ void k_pad(const double* src, double* dst, int ny, int nx, int Py, int Px) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    size_t sl = blockIdx.z;
    if (i >= Px) return;
    double v = (j < ny && i < nx) ? src[sl * (size_t)ny * nx + (size_t)j * nx + i] : 0.0;
    dst[sl * (size_t)Py * Px + (size_t)j * Px + i] = v;
}

template <typename T>
__global__ void k_unpad(const T* src, T* dst, int ny, int nx, int Py, int Px) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    size_t sl = blockIdx.z;
    if (i >= nx) return;
    dst[sl * (size_t)ny * nx + (size_t)j * nx + i] = src[sl * (size_t)Py * Px + (size_t)j * Px + i];
}

// SplitMix64 (Steele, Lea, Flood 2014): output number idx of the generator seeded with `seed`
// is mix(seed + (idx+1) * 0x9E3779B97F4A7C15); mapped to uniform[-1, 1) with 53 bits.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t idx) {
    uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

__global__ void k_fill_random(double* u, int ny, int nx, int Py, int Px, uint64_t seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    size_t n = (size_t)blockIdx.z + 1;  // time index 1..nt
    if (i >= Px) return;
    double v = 0.0;
    if (i < nx && j < ny) v = splitmix_uniform(seed, (n * (size_t)ny + j) * nx + i);
    u[n * (size_t)Py * Px + (size_t)j * Px + i] = v;
}

__global__ void k_axpy_strided(double* y, long long ys, const double* x, long long xs, size_t P2) {
    size_t sl = blockIdx.y;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P2; e += (size_t)gridDim.x * blockDim.x)
        y[sl * ys + e] += x[sl * xs + e];
}

}  // namespace

// ------------------------------------------------------------------------------------------

void sfde_launch_pad(const double* src, double* dst, int ny, int nx, int Py, int Px, int slices,
                     cudaStream_t s) {
    dim3 grid((Px + 127) / 128, Py, slices);
    k_pad<<<grid, 128, 0, s>>>(src, dst, ny, nx, Py, Px);
}

void sfde_launch_unpad(const double* src, double* dst, int ny, int nx, int Py, int Px, int slices,
                       cudaStream_t s) {
    dim3 grid((nx + 127) / 128, ny, slices);
    k_unpad<double><<<grid, 128, 0, s>>>(src, dst, ny, nx, Py, Px);
}

void sfde_launch_unpad_f32(const float* src, float* dst, int ny, int nx, int Py, int Px, int slices,
                           cudaStream_t s) {
    dim3 grid((nx + 127) / 128, ny, slices);
    k_unpad<float><<<grid, 128, 0, s>>>(src, dst, ny, nx, Py, Px);
}

void sfde_launch_fill_random(double* u, int nt, int ny, int nx, int Py, int Px, uint64_t seed,
                             cudaStream_t s) {
    dim3 grid((Px + 127) / 128, Py, nt);
    k_fill_random<<<grid, 128, 0, s>>>(u, ny, nx, Py, Px, seed);
}

void sfde_launch_axpy_strided(double* y, long long y_stride, const double* x, long long x_stride,
                              int slices, size_t P2, cudaStream_t s) {
    dim3 grid((unsigned)((P2 + 255) / 256 < 64 ? (P2 + 255) / 256 : 64), slices);
    k_axpy_strided<<<grid, 256, 0, s>>>(y, y_stride, x, x_stride, P2);
}

// 32, 64, then multiples of 128 so that a 128-row tensor-core tile never straddles two slices
static int pad_dim(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : ((n + 127) / 128) * 128; }

sfde_status sfde_setup_direction(SfdeDir& d, int n, double rho, double length, cudaStream_t s) {
    d.n = n;
    d.P = pad_dim(n);
    d.rho = rho;
    d.h = length / (n + 1);
    const int P = d.P;
    const int ne = n + (n & 1);  // even order for the round-robin pairing
    const double p = 3.0 - 2.0 * rho;
    const double pref = pow(d.h, 1.0 - 2.0 * rho) / (2.0 * cos(rho * M_PI) * tgamma(4.0 - 2.0 * rho));

    size_t PP = (size_t)P * P;
    SFDE_CUDA(cudaMalloc(&d.coeffs, sizeof(double) * n));
    SFDE_CUDA(cudaMalloc(&d.A, sizeof(double) * PP));
    SFDE_CUDA(cudaMalloc(&d.lam, sizeof(double) * P));
    SFDE_CUDA(cudaMalloc(&d.V, sizeof(double) * PP));
    SFDE_CUDA(cudaMalloc(&d.W, sizeof(double) * PP));
    SFDE_CUDA(cudaMalloc(&d.VT, sizeof(double) * PP));
    SFDE_CUDA(cudaMalloc(&d.WT, sizeof(double) * PP));

    k_toeplitz_coeffs<<<(n + 127) / 128, 128, 0, s>>>(d.coeffs, n, p, pref);
    k_toeplitz_dense<<<dim3((P + 127) / 128, P), 128, 0, s>>>(d.coeffs, d.A, n, P);

    // scratch: l, e, Y, C, Q (ne x ne), rotations, norms
    double *l = nullptr, *e = nullptr, *Y = nullptr, *C = nullptr, *Q = nullptr, *nrm = nullptr;
    Rot* rot = nullptr;
    size_t EE = (size_t)ne * ne;
    sfde_status st = SFDE_OK;
    cudaError_t ce = cudaSuccess;
#define SETUP_CUDA(x) do { ce = (x); if (ce != cudaSuccess) { sfde_set_last_cuda_error(ce, #x, __FILE__, __LINE__); st = SFDE_ECUDA; goto done; } } while (0)
    SETUP_CUDA(cudaMalloc(&l, sizeof(double) * ne));
    SETUP_CUDA(cudaMalloc(&e, sizeof(double) * ne));
    SETUP_CUDA(cudaMalloc(&Y, sizeof(double) * EE));
    SETUP_CUDA(cudaMalloc(&C, sizeof(double) * EE));
    SETUP_CUDA(cudaMalloc(&Q, sizeof(double) * EE));
    SETUP_CUDA(cudaMalloc(&rot, sizeof(Rot) * (ne / 2 + 1)));
    SETUP_CUDA(cudaMalloc(&nrm, sizeof(double) * 2));
    SETUP_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * EE, s));
    SETUP_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * EE, s));

    k_mass_cholesky<<<1, 1, 0, s>>>(l, e, n, d.h);
    // A restricted to n x n with leading dimension ne: copy from the padded P x P matrix
    SETUP_CUDA(cudaMemcpy2DAsync(C, sizeof(double) * ne, d.A, sizeof(double) * P, sizeof(double) * n, n,
                                 cudaMemcpyDeviceToDevice, s));
    k_forward_subst_cols<<<(n + 127) / 128, 128, 0, s>>>(C, Y, n, ne, l, e);      // Y = L^{-1} A
    k_forward_subst_rows_T<<<(n + 127) / 128, 128, 0, s>>>(Y, C, n, ne, l, e);    // C = L^{-1} Y^T
    k_symmetrize<<<dim3((ne + 127) / 128, ne), 128, 0, s>>>(C, ne, n);
    k_identity<<<dim3((ne + 127) / 128, ne), 128, 0, s>>>(Q, ne);

    if (ne >= 2 && ne <= JACOBI_SMEM_MAX) {
        // one launch for the whole iteration (C and Q in shared memory)
        SETUP_CUDA(cudaFuncSetAttribute(k_jacobi_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(double) * 2 * JACOBI_SMEM_MAX * JACOBI_SMEM_MAX)));
        k_jacobi_small<<<1, 256, sizeof(double) * 2 * EE, s>>>(C, Q, ne, 30);
    } else if (ne >= 2) {
        double hn[2];
        for (int sweep = 0; sweep < 30; ++sweep) {
            for (int round = 0; round < ne - 1; ++round) {
                k_jacobi_rotations<<<(ne / 2 + 127) / 128, 128, 0, s>>>(C, ne, round, rot);
                k_jacobi_apply<<<dim3((ne / 2 + 127) / 128, ne / 2), 128, 0, s>>>(C, ne, rot);
                k_jacobi_apply_Q<<<dim3((ne / 2 + 127) / 128, ne), 128, 0, s>>>(Q, ne, rot);
            }
            SETUP_CUDA(cudaMemsetAsync(nrm, 0, sizeof(double) * 2, s));
            k_offdiag_norm<<<64, 256, 0, s>>>(C, ne, nrm);
            SETUP_CUDA(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, s));
            SETUP_CUDA(cudaStreamSynchronize(s));
            // off-diagonal mass down to the rounding floor (about n eps^2 of the diagonal)
            if (hn[0] <= 1e-30 * (double)ne * hn[1]) break;
        }
    }
    k_back_subst_eigvec<<<(P + 127) / 128, 128, 0, s>>>(Q, C, ne, n, P, l, e, d.V, d.lam);
    k_mass_apply_cols<<<dim3((P + 127) / 128, P), 128, 0, s>>>(d.V, d.W, n, P, d.h);
    k_transpose<<<dim3(P / 32, P / 32), dim3(32, 8), 0, s>>>(d.V, d.VT, P);
    k_transpose<<<dim3(P / 32, P / 32), dim3(32, 8), 0, s>>>(d.W, d.WT, P);
    SETUP_CUDA(cudaGetLastError());
    SETUP_CUDA(cudaStreamSynchronize(s));
done:
    cudaFree(l); cudaFree(e); cudaFree(Y); cudaFree(C); cudaFree(Q); cudaFree(rot); cudaFree(nrm);
#undef SETUP_CUDA
    return st;
}

void sfde_free_direction(SfdeDir& d) {
    cudaFree(d.coeffs); cudaFree(d.A); cudaFree(d.lam); cudaFree(d.V); cudaFree(d.W);
    cudaFree(d.VT); cudaFree(d.WT); cudaFree(d.V32); cudaFree(d.W32);
    d = SfdeDir();
}

sfde_status sfde_project_forcing(sfde_ctx* c, const double* bx_dev, const double* by_dev) {
    if (c->rank == 0) return SFDE_OK;
    k_project_factor<<<dim3((c->x.P + 127) / 128, c->rank), 128, 0, c->stream>>>(bx_dev, c->x.V, c->px, c->rank, c->x.n, c->x.P);
    k_project_factor<<<dim3((c->y.P + 127) / 128, c->rank), 128, 0, c->stream>>>(by_dev, c->y.V, c->py, c->rank, c->y.n, c->y.P);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}
