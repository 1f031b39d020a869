// Translation operators (Sec. 2.2: the M2M, M2L and L2L operators are
// matrices between surfaces, computed automatically from the kernel).
//
// All operators are built for a unit box (half-width 1) with the kernel 1/r
// (the 1/(4 pi) factor is applied once at the output).  The library keeps
// every expansion as a potential on a check surface, so each operator that
// crosses an equivalent surface is a composite K_target<-equiv * pinv(K_check<-equiv):
//
//   M2M  A_c = 1/2 K(UC_parent, UE_child c) P_up     (u child -> u parent)
//   M2L  M_o = K(DC, UE + 2 d_o) P_up                 (u source -> d target)
//   L2L  C_c = K(DC_child c, DE_parent) P_dn          (d parent -> d child)
//
// where P = V diag(sinv) U^T is the pseudo-inverse of the check-from-
// equivalent matrix, truncated at eps * sigma_max.  The SVD is a one-sided
// Jacobi (Hestenes) iteration in FP64 on the GPU with a cyclic round-robin
// pair order (Brent & Luk); products are formed as ((K V) diag(sinv)) U^T so
// the large entries of P never appear explicitly.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace kifmm {

namespace {

constexpr int kSvdThreads = 512;

// One block per matrix.  At: [n][n] row j = column j of the matrix; on exit
// row j = sigma_j u_j.  Vt: [n][n] row j = column j of V.
__global__ void k_jacobi_svd(int n, double *At_all, double *Vt_all, double *sigma_all, int max_sweeps,
                             double tol, int *sweeps_out) {
    double *At = At_all + (size_t)blockIdx.x * n * n;
    double *Vt = Vt_all + (size_t)blockIdx.x * n * n;
    double *sigma = sigma_all + (size_t)blockIdx.x * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Vt[i] = (i / n == i % n) ? 1.0 : 0.0;
    __shared__ int rotated;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < n - 1; ++r) {
            for (int k = warp; k < n / 2; k += nwarps) {
                const int i = (k == 0) ? 0 : ((r + k - 1) % (n - 1)) + 1;
                const int j = ((r + n - 2 - k) % (n - 1)) + 1;
                double *ai = At + (size_t)i * n, *aj = At + (size_t)j * n;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int row = lane; row < n; row += 32) {
                    const double x = ai[row], y = aj[row];
                    a += x * x;
                    b += y * y;
                    g += x * y;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (g != 0.0 && fabs(g) > tol * sqrt(a * b)) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    for (int row = lane; row < n; row += 32) {
                        const double x = ai[row], y = aj[row];
                        ai[row] = c * x - s * y;
                        aj[row] = s * x + c * y;
                    }
                    double *vi = Vt + (size_t)i * n, *vj = Vt + (size_t)j * n;
                    for (int row = lane; row < n; row += 32) {
                        const double x = vi[row], y = vj[row];
                        vi[row] = c * x - s * y;
                        vj[row] = s * x + c * y;
                    }
                    if (lane == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    for (int j = warp; j < n; j += nwarps) {
        double *aj = At + (size_t)j * n;
        double s2 = 0.0;
        for (int row = lane; row < n; row += 32) s2 += aj[row] * aj[row];
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const double sg = sqrt(s2);
        for (int row = lane; row < n; row += 32) aj[row] = (sg > 0.0) ? aj[row] / sg : 0.0;
        if (lane == 0) sigma[j] = sg;
    }
    if (threadIdx.x == 0) sweeps_out[blockIdx.x] = sweep;
}

// C[b] = scale * A[b] diag(cs) op(B) with op(B)(m, j) = transB ? B[j][m] : B[m][j];
// all n x n row-major FP64; the result is written transposed when transC.
__global__ void k_dgemm(int n, const double *__restrict__ A, size_t strideA, const double *__restrict__ B,
                        const double *__restrict__ cs, int transB, double scale, double *C, size_t strideC,
                        int transC) {
    __shared__ double As[16][17], Bs[16][17];
    const int b = blockIdx.z;
    const double *Ab = A + strideA * b;
    double *Cb = C + strideC * b;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    double acc = 0.0;
    for (int m0 = 0; m0 < n; m0 += 16) {
        const int ma = m0 + threadIdx.x, mb = m0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] = (i < n && ma < n) ? Ab[(size_t)i * n + ma] * (cs ? cs[ma] : 1.0) : 0.0;
        double bv = 0.0;
        if (mb < n && j < n) bv = transB ? B[(size_t)j * n + mb] : B[(size_t)mb * n + j];
        Bs[threadIdx.y][threadIdx.x] = bv;
        __syncthreads();
        for (int m = 0; m < 16; ++m) acc += As[threadIdx.y][m] * Bs[m][threadIdx.x];
        __syncthreads();
    }
    if (i < n && j < n) {
        if (transC) Cb[(size_t)j * n + i] = scale * acc; else Cb[(size_t)i * n + j] = scale * acc;
    }
}

// out[b] = in[map(b)]^T for n x n blocks; map(b) = rev ? nb - 1 - b : b.
__global__ void k_transpose_blocks(int n, int nb, int rev, const double *__restrict__ in, double *__restrict__ out) {
    const size_t nn = (size_t)n * n;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nn * nb) return;
    const int b = (int)(idx / nn);
    const int r = (int)((idx % nn) / n), c = (int)(idx % n);
    const int src = rev ? nb - 1 - b : b;
    out[idx] = in[(size_t)src * nn + (size_t)c * n + r];
}

__global__ void k_to_f32(const double *in, float *out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// W_t[j][m] = sinv[m] * Ut[m][j]
// Split each check-to-check block [k][j] (input k, output j) into its mean
// over the outputs, mean[blk][k] = (1/n) sum_j A[k][j], and the mean-free
// remainder A[k][j] - mean[blk][k].  One thread per (block, k) row.
__global__ void k_center_rows(int n, int nb, double *A, double *mean) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (int64_t)nb * n) return;
    double *row = A + r * n;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += row[j];
    const double m = s / n;
    for (int j = 0; j < n; ++j) row[j] -= m;
    mean[r] = m;
}

// [nb][n][n] mean-free blocks + [nb][n] mean rows -> FP32 [nb][n][n + 1]
// with the mean in column n.
__global__ void k_pack_mean_col(int n, int nb, const double *__restrict__ A, const double *__restrict__ mean,
                                float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ld = n + 1;
    if (i >= (int64_t)nb * n * ld) return;
    const int64_t row = i / ld;  // blk * n + k
    const int j = (int)(i - row * ld);
    out[i] = (float)((j < n) ? A[row * n + j] : mean[row]);
}

__global__ void k_make_wt(int n, const double *Ut, const double *sinv, double *Wt) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int j = idx / n, m = idx % n;
    Wt[idx] = sinv[m] * Ut[(size_t)m * n + j];
}

// G[i][l] = sum_b sum_m A_b[m][i] A_b[m][l]: the Gram matrix of nb row-major
// n x n blocks stacked vertically.  One thread per (i, l).
__global__ void k_gram(int n, int nb, const double *__restrict__ A, double *__restrict__ G) {
    const int i = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double *Ab = A + (size_t)b * n * n;
        for (int m = 0; m < n; ++m) acc += Ab[(size_t)m * n + i] * Ab[(size_t)m * n + l];
    }
    G[(size_t)i * n + l] = acc;
}

// out[b][c] = sum_k mean[b][k] V[k][c] (V row-major n x n, columns >= r zero).
__global__ void k_mean_proj(int n, int nb, const double *__restrict__ mean, const double *__restrict__ V,
                            double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb * n) return;
    const int b = (int)(t / n), c = (int)(t % n);
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += mean[(size_t)b * n + k] * V[(size_t)k * n + c];
    out[t] = acc;
}

// FP32 [nb][rr][rl + 1]: Bt[b][c][i] for i < rl, the mean row mh[b][c] at i = rl.
__global__ void k_pack_compressed(int n, int nb, int rr, int rl, const double *__restrict__ Bt,
                                  const double *__restrict__ mh, float *__restrict__ out) {
    const int64_t ld = rl + 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb * rr * ld) return;
    const int b = (int)(t / (rr * ld));
    const int c = (int)((t / ld) % rr), i = (int)(t % ld);
    out[t] = (float)((i < rl) ? Bt[((size_t)b * n + c) * n + i] : mh[(size_t)b * n + c]);
}


// K[i][k] = 1 / |(ct + at S_i) - (cs + as S_k)|
void kernel_block(const std::vector<double> &S, int n, const double ct[3], double at, const double cs[3],
                  double as, double *K) {
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double dd = (ct[d] + at * S[3 * i + d]) - (cs[d] + as * S[3 * k + d]);
                r2 += dd * dd;
            }
            K[(size_t)i * n + k] = (r2 > 0.0) ? 1.0 / std::sqrt(r2) : 0.0;
        }
}

// The Stokeslet block of the same surfaces (the tensor kernel of Eq. 1, Sec.
// 2.4's Stokes flow): [3 n][3 n], row 3 i + a, column 3 k + b holds
// G_ab(r) = delta_ab / |r| + r_a r_b / |r|^3 (the 1 / (8 pi mu) is applied
// with coef), r = target_i - source_k; zero at r = 0.
void stokes_block(const std::vector<double> &S, int n, const double ct[3], double at, const double cs[3], double as,
                  double *K) {
    const size_t ld = 3 * (size_t)n;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double r[3], r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                r[d] = (ct[d] + at * S[3 * i + d]) - (cs[d] + as * S[3 * k + d]);
                r2 += r[d] * r[d];
            }
            const double ri = (r2 > 0.0) ? 1.0 / std::sqrt(r2) : 0.0, ri3 = ri * ri * ri;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    K[(3 * (size_t)i + a) * ld + 3 * k + b] = (a == b ? ri : 0.0) + r[a] * r[b] * ri3;
        }
}

void child_center(int o, double c[3]) {
    c[0] = ((o >> 2) & 1) ? 0.5 : -0.5;
    c[1] = ((o >> 1) & 1) ? 0.5 : -0.5;
    c[2] = (o & 1) ? 0.5 : -0.5;
}

}  // namespace

// Unit-cube surface grid (half-width 1): p points per edge, the boundary
// points of the p^3 lattice in lexicographic order, n_s = 6 (p - 1)^2 + 2.
std::vector<double> unit_surface(int p) {
    std::vector<double> s;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                if (i == 0 || i == p - 1 || j == 0 || j == p - 1 || k == 0 || k == p - 1) {
                    s.push_back(-1.0 + 2.0 * i / (p - 1));
                    s.push_back(-1.0 + 2.0 * j / (p - 1));
                    s.push_back(-1.0 + 2.0 * k / (p - 1));
                }
            }
    return s;
}

std::vector<int> m2l_offset_list() {
    std::vector<int> out;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1 && c >= -1 && c <= 1) continue;
                out.push_back(a);
                out.push_back(b);
                out.push_back(c);
            }
    return out;
}

// Rank from descending singular values: the count above eps * sig[0],
// rounded up so that rank + mean_slot fills 32-wide tiles (at most n), then
// lowered while the cut would split a cluster (sig[r-1] <= 1.001 sig[r]).
static int compress_rank(const std::vector<double> &sig, double eps, int mean_slot) {
    const int n = (int)sig.size();
    int r0 = 0;
    for (int i = 0; i < n; ++i) r0 += (sig[i] > eps * sig[0]) ? 1 : 0;
    int r = std::min(n, 32 * ((r0 + mean_slot + 31) / 32) - mean_slot);
    while (r > 1 && r < n && sig[r - 1] <= 1.001 * sig[r]) --r;
    return r;
}

// Compressed M2L on shared bases.  K (device): the 316 raw M2L blocks,
// row-major [j][k] (output DC point j, input UE point k).  U: leading
// eigenvectors of sum_o K0_o K0_o^T (K0 = K minus its mean over j); V: of
// sum_o K_o^T K_o; both from the FP64 Jacobi SVD of the symmetric Gram
// matrices (singular values = eigenvalues; the accumulated rotations are the
// eigenvectors).  Builds m2l_c (C_o^T = (U^T K0_o V)^T with the mean row
// m_o^T V in column rl), m2l_wc = V^T P_up and m2l_ul = U, all FP32.
static cudaError_t build_m2l_compressed(Plan &P, const double *dK, const double *Ut_up, const double *Vt_up,
                                        const double *sinv_up, std::string &err) {
    const int n = P.ns;
    const size_t nn = (size_t)n * n;
    const int nb = kNumM2L;
    double *T = nullptr, *mean = nullptr, *K0 = nullptr, *G = nullptr, *Gv = nullptr, *Gs = nullptr;
    int *sw = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&T, sizeof(double) * nb * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&K0, sizeof(double) * nb * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&mean, sizeof(double) * nb * n));
    KIFMM_CUDA_TRY(cudaMalloc(&G, sizeof(double) * 2 * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&Gv, sizeof(double) * 2 * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&Gs, sizeof(double) * 2 * n));
    KIFMM_CUDA_TRY(cudaMalloc(&sw, sizeof(int) * 2));
    const size_t tot = nn * nb;
    // T = K^T ([k][j]); centre each row over j: T0 = K0^T and the means m_o[k]
    k_transpose_blocks<<<(unsigned)((tot + 255) / 256), 256>>>(n, nb, 0, dK, T);
    k_center_rows<<<(unsigned)((nb * n + 255) / 256), 256>>>(n, nb, T, mean);
    // G_L = sum T0^T T0 = sum K0 K0^T; G_R = sum K^T K
    k_gram<<<dim3((n + 127) / 128, n), 128>>>(n, nb, T, G);
    k_gram<<<dim3((n + 127) / 128, n), 128>>>(n, nb, dK, G + nn);
    k_jacobi_svd<<<2, kSvdThreads>>>(n, G, Gv, Gs, 60, 1e-15, sw);
    KIFMM_CUDA_TRY(cudaGetLastError());
    std::vector<double> lam(2 * n), vt(2 * nn);
    int sweeps[2];
    KIFMM_CUDA_TRY(cudaMemcpy(lam.data(), Gs, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
    KIFMM_CUDA_TRY(cudaMemcpy(vt.data(), Gv, sizeof(double) * 2 * nn, cudaMemcpyDeviceToHost));
    KIFMM_CUDA_TRY(cudaMemcpy(sweeps, sw, sizeof(int) * 2, cudaMemcpyDeviceToHost));
    if (sweeps[0] >= 60 || sweeps[1] >= 60) {
        err = "Jacobi eigensolver of the M2L Gram matrices did not converge";
        return cudaErrorUnknown;
    }
    // sort each spectrum (descending) and pick the ranks
    int rank[2];
    std::vector<int> order[2];
    for (int m = 0; m < 2; ++m) {
        order[m].resize(n);
        for (int i = 0; i < n; ++i) order[m][i] = i;
        std::stable_sort(order[m].begin(), order[m].end(),
                         [&](int a, int b) { return lam[m * n + a] > lam[m * n + b]; });
        std::vector<double> sig(n);
        for (int i = 0; i < n; ++i) sig[i] = std::sqrt(std::fmax(lam[m * n + order[m][i]], 0.0));
        rank[m] = compress_rank(sig, P.desc.m2l_eps, m == 0 ? 1 : 0);
    }
    const int rl = rank[0], rr = rank[1];
    // bases, zero-padded to n x n: Up[j][i] = u_i[j] (i < rl); Vp[k][c] = v_c[k] (c < rr)
    std::vector<double> Up(nn, 0.0), Vp(nn, 0.0), VpT(nn, 0.0);
    for (int i = 0; i < rl; ++i)
        for (int j = 0; j < n; ++j) Up[(size_t)j * n + i] = vt[(size_t)order[0][i] * n + j];
    for (int c = 0; c < rr; ++c)
        for (int k = 0; k < n; ++k) {
            Vp[(size_t)k * n + c] = vt[nn + (size_t)order[1][c] * n + k];
            VpT[(size_t)c * n + k] = Vp[(size_t)k * n + c];
        }
    double *dUp = nullptr, *dVp = nullptr, *dVpT = nullptr, *KVt = nullptr, *Bt = nullptr, *mh = nullptr,
           *Y = nullptr, *Wc = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&dUp, sizeof(double) * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dVp, sizeof(double) * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dVpT, sizeof(double) * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&KVt, sizeof(double) * nb * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&Bt, sizeof(double) * nb * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&mh, sizeof(double) * nb * n));
    KIFMM_CUDA_TRY(cudaMalloc(&Y, sizeof(double) * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&Wc, sizeof(double) * nn));
    KIFMM_CUDA_TRY(cudaMemcpy(dUp, Up.data(), sizeof(double) * nn, cudaMemcpyHostToDevice));
    KIFMM_CUDA_TRY(cudaMemcpy(dVp, Vp.data(), sizeof(double) * nn, cudaMemcpyHostToDevice));
    KIFMM_CUDA_TRY(cudaMemcpy(dVpT, VpT.data(), sizeof(double) * nn, cudaMemcpyHostToDevice));
    const dim3 blk(16, 16), grd((n + 15) / 16, (n + 15) / 16, nb), grd1((n + 15) / 16, (n + 15) / 16, 1);
    // K0 row-major, then (K0 V)^T, then Bt = (K0 V)^T U = C^T ([c][i])
    k_transpose_blocks<<<(unsigned)((tot + 255) / 256), 256>>>(n, nb, 0, T, K0);
    k_dgemm<<<grd, blk>>>(n, K0, nn, dVp, nullptr, 0, 1.0, KVt, nn, 1);
    k_dgemm<<<grd, blk>>>(n, KVt, nn, dUp, nullptr, 0, 1.0, Bt, nn, 0);
    k_mean_proj<<<(unsigned)((nb * n + 255) / 256), 256>>>(n, nb, mean, dVp, mh);
    // W = V^T P_up = (V^T V_up) diag(sinv) U_up^T
    k_dgemm<<<grd1, blk>>>(n, dVpT, 0, Vt_up, nullptr, 1, 1.0, Y, 0, 0);
    k_dgemm<<<grd1, blk>>>(n, Y, 0, Ut_up, sinv_up, 0, 1.0, Wc, 0, 0);
    KIFMM_CUDA_TRY(cudaGetLastError());
    const size_t nc = (size_t)nb * rr * (rl + 1);
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.m2l_c, sizeof(float) * nc));
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.m2l_wc, sizeof(float) * (size_t)rr * n));
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.m2l_ul, sizeof(float) * (size_t)n * rl));
    k_pack_compressed<<<(unsigned)((nc + 255) / 256), 256>>>(n, nb, rr, rl, Bt, mh, P.m2l_c);
    k_to_f32<<<(unsigned)(((size_t)rr * n + 255) / 256), 256>>>(Wc, P.m2l_wc, (size_t)rr * n);  // rows < rr
    std::vector<float> ul((size_t)n * rl);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < rl; ++i) ul[(size_t)j * rl + i] = (float)Up[(size_t)j * n + i];
    KIFMM_CUDA_TRY(cudaMemcpy(P.m2l_ul, ul.data(), sizeof(float) * ul.size(), cudaMemcpyHostToDevice));
    KIFMM_CUDA_TRY(cudaDeviceSynchronize());
    P.m2l_rl = rl;
    P.m2l_rr = rr;
    for (double *q : {T, K0, mean, G, Gv, Gs, dUp, dVp, dVpT, KVt, Bt, mh, Y, Wc}) cudaFree(q);
    cudaFree(sw);
    return cudaGetLastError();
}

cudaError_t build_operators(Plan &P, std::string &err) {
    // n: length of a box's expansion vector (n_s for the Laplace kernel, 3 n_s
    // for the Stokeslet's 3-vector densities); ns_pts: surface points
    const int p = P.p, n = P.ns, ns_pts = P.nsurf;
    const std::vector<double> S = unit_surface(p);
    const double zero[3] = {0, 0, 0};
    const size_t nn = (size_t)n * n;
    const double ai = kAlphaInner, ao = kAlphaOuter;
    auto kernel_block = [&](const std::vector<double> &S_, int, const double ct[3], double at, const double cs[3],
                            double as, double *K) {
        if (P.stokes) stokes_block(S_, ns_pts, ct, at, cs, as, K);
        else kifmm::kernel_block(S_, ns_pts, ct, at, cs, as, K);
    };

    // check-from-equivalent matrices, transposed for the column-wise Jacobi
    std::vector<double> Kchk(2 * nn), tmp(nn);
    kernel_block(S, n, zero, ao, zero, ai, tmp.data());  // K(UC, UE)
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) Kchk[(size_t)k * n + i] = tmp[(size_t)i * n + k];
    kernel_block(S, n, zero, ai, zero, ao, tmp.data());  // K(DC, DE)
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) Kchk[nn + (size_t)k * n + i] = tmp[(size_t)i * n + k];

    double *dAt = nullptr, *dVt = nullptr, *dsig = nullptr, *dsinv = nullptr;
    int *dsweeps = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&dAt, sizeof(double) * 2 * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dVt, sizeof(double) * 2 * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dsig, sizeof(double) * 2 * n));
    KIFMM_CUDA_TRY(cudaMalloc(&dsinv, sizeof(double) * 2 * n));
    KIFMM_CUDA_TRY(cudaMalloc(&dsweeps, sizeof(int) * 2));
    KIFMM_CUDA_TRY(cudaMemcpy(dAt, Kchk.data(), sizeof(double) * 2 * nn, cudaMemcpyHostToDevice));
    k_jacobi_svd<<<2, kSvdThreads>>>(n, dAt, dVt, dsig, 60, 1e-15, dsweeps);
    KIFMM_CUDA_TRY(cudaGetLastError());
    std::vector<double> sig(2 * n);
    int sweeps[2];
    KIFMM_CUDA_TRY(cudaMemcpy(sig.data(), dsig, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
    KIFMM_CUDA_TRY(cudaMemcpy(sweeps, dsweeps, sizeof(int) * 2, cudaMemcpyDeviceToHost));
    if (sweeps[0] >= 60 || sweeps[1] >= 60) {
        err = "Jacobi SVD did not converge";
        return cudaErrorUnknown;
    }
    // Truncation.  In FP64 mode the threshold must not lie within a factor 1.1
    // of any sigma_i / sigma_max (the gap check), so that this Jacobi SVD and
    // any other backward-stable SVD truncate the same modes; the FP32-based
    // modes only need some consistent regularisation and skip the check.
    std::vector<double> sinv(2 * n);
    for (int m = 0; m < 2; ++m) {
        double smax = 0.0;
        for (int j = 0; j < n; ++j) smax = std::fmax(smax, sig[m * n + j]);
        for (int j = 0; j < n; ++j) {
            const double rel = sig[m * n + j] / smax;
            if (P.f64 && rel > P.eps / 1.1 && rel < P.eps * 1.1) {
                char buf[160];
                snprintf(buf, sizeof buf, "pinv_eps %.3g lies within a factor 1.1 of sigma/sigma_max = %.3g",
                         P.eps, rel);
                err = buf;
                return cudaErrorInvalidValue;
            }
            sinv[m * n + j] = (rel >= P.eps) ? 1.0 / sig[m * n + j] : 0.0;
        }
    }
    KIFMM_CUDA_TRY(cudaMemcpy(dsinv, sinv.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice));

    // kernel blocks: 8 M2M, 8 L2L, 316 M2L (row-major)
    const std::vector<int> offs = m2l_offset_list();
    const int nblk = 8 + 8 + kNumM2L;
    std::vector<double> Kb((size_t)nblk * nn);
    for (int o = 0; o < 8; ++o) {
        double cc[3];
        child_center(o, cc);
        kernel_block(S, n, zero, ao, cc, 0.5 * ai, Kb.data() + (size_t)o * nn);        // K(UC_p, UE_c)
        kernel_block(S, n, cc, 0.5 * ai, zero, ao, Kb.data() + (size_t)(8 + o) * nn);  // K(DC_c, DE_p)
    }
    for (int o = 0; o < kNumM2L; ++o) {
        const double cs[3] = {2.0 * offs[3 * o], 2.0 * offs[3 * o + 1], 2.0 * offs[3 * o + 2]};
        kernel_block(S, n, zero, ai, cs, ai, Kb.data() + (size_t)(16 + o) * nn);       // K(DC, UE + 2d)
    }
    double *dK = nullptr, *dKV = nullptr, *dOut = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&dK, sizeof(double) * nblk * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dKV, sizeof(double) * nblk * nn));
    KIFMM_CUDA_TRY(cudaMalloc(&dOut, sizeof(double) * nblk * nn));
    KIFMM_CUDA_TRY(cudaMemcpy(dK, Kb.data(), sizeof(double) * nblk * nn, cudaMemcpyHostToDevice));
    const double *Ut_up = dAt, *Ut_dn = dAt + nn, *Vt_up = dVt, *Vt_dn = dVt + nn;
    const double *sinv_up = dsinv, *sinv_dn = dsinv + n;
    dim3 blk(16, 16);
    auto gemm = [&](const double *A, int batch, const double *B, const double *cs, int transB, double scale,
                    double *C, int transC) {
        dim3 grd((n + 15) / 16, (n + 15) / 16, batch);
        k_dgemm<<<grd, blk>>>(n, A, nn, B, cs, transB, scale, C, nn, transC);
    };
    // K V  (V(k, m) = Vt[m][k])
    gemm(dK, 8, Vt_up, nullptr, 1, 1.0, dKV, 0);
    gemm(dK + 8 * nn, 8, Vt_dn, nullptr, 1, 1.0, dKV + 8 * nn, 0);
    gemm(dK + 16 * nn, kNumM2L, Vt_up, nullptr, 1, 1.0, dKV + 16 * nn, 0);
    // (K V) diag(sinv) U^T, written transposed ([k][j]); M2M carries h_child / h_parent = 1/2
    gemm(dKV, 8, Ut_up, sinv_up, 0, 0.5, dOut, 1);
    gemm(dKV + 8 * nn, 8, Ut_dn, sinv_dn, 0, 1.0, dOut + 8 * nn, 1);
    gemm(dKV + 16 * nn, kNumM2L, Ut_up, sinv_up, 0, 1.0, dOut + 16 * nn, 1);
    // leaf pseudo-inverses: W_t = (diag(sinv) U^T)^T, V_t = V^T (stored as is)
    double *dW = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&dW, sizeof(double) * 2 * nn));
    k_make_wt<<<(unsigned)((nn + 255) / 256), 256>>>(n, Ut_up, sinv_up, dW);
    k_make_wt<<<(unsigned)((nn + 255) / 256), 256>>>(n, Ut_dn, sinv_dn, dW + nn);
    KIFMM_CUDA_TRY(cudaGetLastError());

    const size_t esz = P.f64 ? sizeof(double) : sizeof(float);
    KIFMM_CUDA_TRY(plan_alloc(P, &P.m2m_t, esz * 8 * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.l2l_t, esz * 8 * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.m2l_t, esz * kNumM2L * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.up_w_t, esz * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.up_v_t, esz * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.dn_w_t, esz * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.dn_v_t, esz * nn));
    struct Copy { void *dst; const double *src; size_t cnt; };
    const Copy copies[] = {{P.m2m_t, dOut, 8 * nn},           {P.l2l_t, dOut + 8 * nn, 8 * nn},
                           {P.m2l_t, dOut + 16 * nn, kNumM2L * nn}, {P.up_w_t, dW, nn},
                           {P.up_v_t, Vt_up, nn},             {P.dn_w_t, dW + nn, nn},
                           {P.dn_v_t, Vt_dn, nn}};
    for (const Copy &c : copies) {
        if (P.f64)
            KIFMM_CUDA_TRY(cudaMemcpy(c.dst, c.src, sizeof(double) * c.cnt, cudaMemcpyDeviceToDevice));
        else
            k_to_f32<<<(unsigned)((c.cnt + 255) / 256), 256>>>(c.src, (float *)c.dst, c.cnt);
    }
    if (!P.stokes) {
    // Adjoint operators (the transposed passes use the same gathered GEMM, which
    // reads operators as [k][j]; for Op^T that is Op itself, row-major):
    //   M2M^T, L2L^T: blocks of m2m_t / l2l_t transposed back;
    //   M2L^T at offset o: M_{-o} row-major, and -o has index 315 - o.
    //   Leaf pseudo-inverses W^T, V^T: W and V row-major.
    double *dT = nullptr;
    KIFMM_CUDA_TRY(cudaMalloc(&dT, sizeof(double) * (size_t)(16 + kNumM2L + 4) * nn));
    auto tblocks = [&](const double *in, int nb, int rev, double *out) {
        const size_t tot = nn * nb;
        k_transpose_blocks<<<(unsigned)((tot + 255) / 256), 256>>>(n, nb, rev, in, out);
    };
    tblocks(dOut, 8, 0, dT);                             // m2m row-major
    tblocks(dOut + 8 * nn, 8, 0, dT + 8 * nn);           // l2l row-major
    tblocks(dOut + 16 * nn, kNumM2L, 1, dT + 16 * nn);   // m2l at negated offsets, row-major
    tblocks(dW, 1, 0, dT + (16 + kNumM2L) * nn);         // up W row-major
    tblocks(Vt_up, 1, 0, dT + (17 + kNumM2L) * nn);      // up V row-major
    tblocks(dW + nn, 1, 0, dT + (18 + kNumM2L) * nn);    // dn W row-major
    tblocks(Vt_dn, 1, 0, dT + (19 + kNumM2L) * nn);      // dn V row-major
    KIFMM_CUDA_TRY(plan_alloc(P, &P.adj_m2m, esz * 8 * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.adj_l2l, esz * 8 * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.adj_m2l, esz * kNumM2L * nn));
    KIFMM_CUDA_TRY(plan_alloc(P, &P.adj_pinv, esz * 4 * nn));
    const Copy adj[] = {{P.adj_m2m, dT, 8 * nn},
                        {P.adj_l2l, dT + 8 * nn, 8 * nn},
                        {P.adj_m2l, dT + 16 * nn, kNumM2L * nn},
                        {P.adj_pinv, dT + (16 + kNumM2L) * nn, 4 * nn}};
    for (const Copy &c : adj) {
        if (P.f64)
            KIFMM_CUDA_TRY(cudaMemcpy(c.dst, c.src, sizeof(double) * c.cnt, cudaMemcpyDeviceToDevice));
        else
            k_to_f32<<<(unsigned)((c.cnt + 255) / 256), 256>>>(c.src, (float *)c.dst, c.cnt);
    }
    KIFMM_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(dT);
    }  // adjoint operators (Laplace)
    P.op_ld = n;
    if (!P.f64 && !P.stokes) {
        // FP32-based modes carry the downward check potential as a per-box
        // mean (FP64 scalar) plus a mean-free FP32 vector: the L2L and M2L
        // blocks are stored mean-free, [k][n + 1] with the mean row in
        // column n, so the same GEMMs produce the mean contributions.
        double *dMean = nullptr;
        KIFMM_CUDA_TRY(cudaMalloc(&dMean, sizeof(double) * (8 + kNumM2L) * n));
        const int64_t rows = (int64_t)(8 + kNumM2L) * n;
        k_center_rows<<<(unsigned)((rows + 255) / 256), 256>>>(n, 8 + kNumM2L, dOut + 8 * nn, dMean);
        P.op_ld = n + 1;
        const size_t blk1 = (size_t)n * (n + 1);
        KIFMM_CUDA_TRY(plan_alloc(P, &P.l2l_t, sizeof(float) * 8 * blk1));
        KIFMM_CUDA_TRY(plan_alloc(P, &P.m2l_t, sizeof(float) * kNumM2L * blk1));
        k_pack_mean_col<<<(unsigned)((8 * blk1 + 255) / 256), 256>>>(n, 8, dOut + 8 * nn, dMean, (float *)P.l2l_t);
        k_pack_mean_col<<<(unsigned)((kNumM2L * blk1 + 255) / 256), 256>>>(n, kNumM2L, dOut + 16 * nn, dMean + 8 * n,
                                                                         (float *)P.m2l_t);
        KIFMM_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(dMean);
    }
    if (P.desc.m2l_eps > 0.0) KIFMM_CUDA_TRY(build_m2l_compressed(P, dK + 16 * nn, Ut_up, Vt_up, sinv_up, err));
    if (P.periodic) {
        // Periodic cell (Sec. 2.4).  Far images on the root: K_far is the
        // far-image matrix (root DC <- root UE over the images beyond the 26
        // nearest) for the unit box (half-width 1, cell side 2) in this
        // library's kernel 1/r; the composite F = K_far V diag(sinv) U^T maps
        // the root's upward check potential to its downward one, like an M2L
        // block, and is stored transposed ([k][j]) in the compute type.
        std::vector<double> T(nn);
        KIFMM_CUDA_TRY(far_image_operator(p, 2.0, T.data()));
        for (double &v : T) v *= 4.0 * 3.14159265358979323846;
        double *dKf = nullptr, *dKfV = nullptr, *dF = nullptr;
        KIFMM_CUDA_TRY(cudaMalloc(&dKf, sizeof(double) * nn));
        KIFMM_CUDA_TRY(cudaMalloc(&dKfV, sizeof(double) * nn));
        KIFMM_CUDA_TRY(cudaMalloc(&dF, sizeof(double) * nn));
        KIFMM_CUDA_TRY(cudaMemcpy(dKf, T.data(), sizeof(double) * nn, cudaMemcpyHostToDevice));
        gemm(dKf, 1, Vt_up, nullptr, 1, 1.0, dKfV, 0);
        gemm(dKfV, 1, Ut_up, sinv_up, 0, 1.0, dF, 1);
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.far_t, sizeof(double) * nn));
        KIFMM_CUDA_TRY(cudaMemcpy(P.far_t, dF, sizeof(double) * nn, cudaMemcpyDeviceToDevice));
        if (!P.f64) {
            // FP32-based modes: the root sums the whole neutral cell, whose
            // contributions cancel; its upward check potential is formed in
            // FP64 from the level-1 boxes (M2M composites kept in FP64)
            KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.m2m64, sizeof(double) * 8 * nn));
            KIFMM_CUDA_TRY(cudaMemcpy(P.m2m64, dOut, sizeof(double) * 8 * nn, cudaMemcpyDeviceToDevice));
            KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.u_root64, sizeof(double) * n));
        }
        // Second-moment functional of the root: the root's equivalent density
        // (half-width h = 1/2 of the unit root) is h P u with P = V diag(sinv)
        // U^T, on the points 1.05 h S_k, so the trace of its second moment
        // about the centre is g . u with g_j = h (1.05 h)^2 sum_k P[k][j] |S_k|^2.
        std::vector<double> Vt(nn), Ut(nn), si(n);
        KIFMM_CUDA_TRY(cudaMemcpy(Vt.data(), Vt_up, sizeof(double) * nn, cudaMemcpyDeviceToHost));
        KIFMM_CUDA_TRY(cudaMemcpy(Ut.data(), Ut_up, sizeof(double) * nn, cudaMemcpyDeviceToHost));
        KIFMM_CUDA_TRY(cudaMemcpy(si.data(), sinv_up, sizeof(double) * n, cudaMemcpyDeviceToHost));
        std::vector<double> am(n, 0.0), g(n, 0.0);
        for (int m = 0; m < n; ++m)  // a_m = sum_k V[k][m] |S_k|^2, V[k][m] = Vt[m][k]
            for (int k = 0; k < n; ++k)
                am[m] += Vt[(size_t)m * n + k] * (S[3 * k] * S[3 * k] + S[3 * k + 1] * S[3 * k + 1] + S[3 * k + 2] * S[3 * k + 2]);
        const double h = 0.5, rz = kAlphaInner * h;
        for (int j = 0; j < n; ++j) {  // U[j][m] = Ut[m][j]
            double acc = 0.0;
            for (int m = 0; m < n; ++m) acc += si[m] * Ut[(size_t)m * n + j] * am[m];
            g[j] = h * rz * rz * acc;
        }
        KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.far_g, sizeof(double) * n));
        KIFMM_CUDA_TRY(cudaMemcpy(P.far_g, g.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        KIFMM_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(dKf);
        cudaFree(dKfV);
        cudaFree(dF);
    }
    // surfaces
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.surf64, sizeof(double) * 3 * ns_pts));
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.surf32, sizeof(float) * 3 * ns_pts));
    std::vector<float> S32(S.begin(), S.end());
    KIFMM_CUDA_TRY(cudaMemcpy(P.surf64, S.data(), sizeof(double) * 3 * ns_pts, cudaMemcpyHostToDevice));
    KIFMM_CUDA_TRY(cudaMemcpy(P.surf32, S32.data(), sizeof(float) * 3 * ns_pts, cudaMemcpyHostToDevice));
    // V slot -> offset index tables
    std::vector<int> slot(8 * kVSlots, -1);
    for (int cls = 0; cls < 8; ++cls) {
        const int ox = (cls >> 2) & 1, oy = (cls >> 1) & 1, oz = cls & 1;
        int s = 0;
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b)
                for (int c = 0; c < 6; ++c) {
                    const int dx = a - 2 - ox, dy = b - 2 - oy, dz = c - 2 - oz;
                    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) continue;
                    int idx = 0;
                    for (int t = 0; t < kNumM2L; ++t)
                        if (offs[3 * t] == dx && offs[3 * t + 1] == dy && offs[3 * t + 2] == dz) idx = t;
                    slot[cls * kVSlots + s++] = idx;
                }
    }
    KIFMM_CUDA_TRY(plan_alloc(P, (void **)&P.slot_off, sizeof(int) * 8 * kVSlots));
    KIFMM_CUDA_TRY(cudaMemcpy(P.slot_off, slot.data(), sizeof(int) * 8 * kVSlots, cudaMemcpyHostToDevice));
    KIFMM_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(dAt);
    cudaFree(dVt);
    cudaFree(dsig);
    cudaFree(dsinv);
    cudaFree(dsweeps);
    cudaFree(dK);
    cudaFree(dKV);
    cudaFree(dOut);
    cudaFree(dW);
    return cudaGetLastError();
}

}  // namespace kifmm
