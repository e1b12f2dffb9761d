// ba.cu -- one Levenberg-Marquardt step of the tracker's dense visual bundle
// adjustment (Sec. 3.2: vision residual Eq. 2 over the edges of the frame graph,
// normal equations solved by the Schur complement of the diagonal depth block,
// Eq. 4).
//
//   r = u*_ij - Pi(T_j T_i^-1 Pi^-1(u, d_i(u)))  for every edge (i, j) and pixel u
//   of keyframe i; cost sum w r^2.  Variables: left perturbations xi_k = (rho, phi)
//   of the poses k >= n_fixed (T_k <- Exp(xi_k) T_k) and every inverse depth.
//   With p = R_ij xbar + d t_ij (the point times its inverse depth):
//     dp/d rho_j = d I, dp/d phi_j = -[p]x,  dp/d rho_i = -d R_ij,
//     dp/d phi_i = R_ij [xbar]x,  dp/d d = t_ij.
//   H = [B E; E^T C] with C diagonal (a residual depends on one inverse depth);
//   (B + damping - E C'^-1 E^T) dxi = -g_xi + E C'^-1 g_d,
//   dd = C'^-1 (-g_d - E^T dxi),  C' = (1 + lambda) C + eps.
//
// Kernels: k_ba_terms (one thread per (edge, pixel): residual, Jacobians, B and
// g_xi reduced per CTA into dense buffers, C and g_d by atomics, the 12-vector
// E(e, p) = [J_i^T W J_d, J_j^T W J_d] stored), k_ba_damp (diagonal damping of
// B), k_ba_schur (one CTA per ordered pair of edges with the same source
// keyframe: sum_p E(e1, p) E(e2, p)^T / C'_p into the four 6x6 blocks it touches,
// and E C'^-1 g_d into the right-hand side), k_ba_solve (one CTA: Cholesky of
// the n x n reduced system in shared memory), k_ba_update (inverse depths by
// back-substitution, poses by Exp).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kTermThreads = 128;
constexpr int kTermVals = 21 + 36 + 21 + 6 + 6 + 1;   // H_ii (upper), H_ij, H_jj (upper), g_i, g_j, cost

struct BaDev {
    float* poses;          // [K][12]
    float* disp;           // [K][P]
    const float* targets;  // [E][P][2]
    const float* weights;  // [E][P][2]
    const int32_t* ii;
    const int32_t* jj;
    int K, E, h, w, P, n_fixed, n;   // n = 6 (K - n_fixed)
    float fx, fy, cx, cy;
    float* Eb;             // [E][P][12]
    float* C;              // [K][P]
    float* gd;             // [K][P]
    float* S;              // [n][n]
    float* rhs;            // [n]
    float* dxi;            // [n]
    float* cost;           // [1]
    int* status;
};

__device__ __forceinline__ bool edge_ok(const BaDev& b, int i, int j) {
    return i >= 0 && i < b.K && j >= 0 && j < b.K && i != j;
}

__device__ __forceinline__ void rel_pose(const BaDev& b, int i, int j, float* Rij, float* tij) {
    const float* Pi = b.poses + 12 * i;
    const float* Pj = b.poses + 12 * j;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Rij[3 * r + c] = Pj[3 * r] * Pi[3 * c] + Pj[3 * r + 1] * Pi[3 * c + 1] + Pj[3 * r + 2] * Pi[3 * c + 2];
    for (int r = 0; r < 3; r++)
        tij[r] = Pj[9 + r] - (Rij[3 * r] * Pi[9] + Rij[3 * r + 1] * Pi[10] + Rij[3 * r + 2] * Pi[11]);
}

// sum over the CTA of kTermVals values per thread; thread t < kTermVals gets total t
__device__ __forceinline__ float block_sum_vals(float (&v)[kTermVals], float* s_part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kTermVals; k++) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_part[warp * kTermVals + k] = x;
    }
    __syncthreads();
    float tot = 0.f;
    if ((int)threadIdx.x < kTermVals)
        for (int w = 0; w < kTermThreads / 32; w++) tot += s_part[w * kTermVals + threadIdx.x];
    return tot;
}

__global__ void __launch_bounds__(kTermThreads) k_ba_terms(BaDev b) {
    __shared__ float s_part[(kTermThreads / 32) * kTermVals];
    const int e = blockIdx.y;
    const int q = blockIdx.x * kTermThreads + threadIdx.x;
    const int i = b.ii[e], j = b.jj[e];
    float v[kTermVals];
#pragma unroll
    for (int k = 0; k < kTermVals; k++) v[k] = 0.f;
    if (!edge_ok(b, i, j)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(b.status, 0, GS_ERR_INVALID_ARG);
        return;   // the whole CTA returns: no barrier is reached
    }
    if (q < b.P) {
        float Rij[9], tij[3];
        rel_pose(b, i, j, Rij, tij);
        const int y = q / b.w, x = q % b.w;
        const float xb[3] = {((float)x + 0.5f - b.cx) / b.fx, ((float)y + 0.5f - b.cy) / b.fy, 1.0f};
        const float d = b.disp[(size_t)i * b.P + q];
        float p[3];
        for (int r = 0; r < 3; r++) p[r] = Rij[3 * r] * xb[0] + Rij[3 * r + 1] * xb[1] + Rij[3 * r + 2] * xb[2] + d * tij[r];
        const float iz = 1.0f / p[2];
        const size_t o = ((size_t)e * b.P + q) * 2;
        const float r0 = b.targets[o] - (b.fx * p[0] * iz + b.cx);
        const float r1 = b.targets[o + 1] - (b.fy * p[1] * iz + b.cy);
        const float w0 = b.weights[o], w1 = b.weights[o + 1];
        // dr/dp = -dPi/dp
        const float a00 = -b.fx * iz, a02 = b.fx * p[0] * iz * iz;
        const float a11 = -b.fy * iz, a12 = b.fy * p[1] * iz * iz;
        // dp/d(xi_j) = [d I, -[p]x], dp/d(xi_i) = [-d R_ij, R_ij [xb]x]
        float Dj[3][6], Di[3][6];
        const float pk[3][3] = {{0.f, p[2], -p[1]}, {-p[2], 0.f, p[0]}, {p[1], -p[0], 0.f}};      // -[p]x
        const float xk[3][3] = {{0.f, -xb[2], xb[1]}, {xb[2], 0.f, -xb[0]}, {-xb[1], xb[0], 0.f}}; // [xb]x
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                Dj[r][c] = r == c ? d : 0.f;
                Dj[r][3 + c] = pk[r][c];
                Di[r][c] = -d * Rij[3 * r + c];
                Di[r][3 + c] = Rij[3 * r] * xk[0][c] + Rij[3 * r + 1] * xk[1][c] + Rij[3 * r + 2] * xk[2][c];
            }
        float Ji[2][6], Jj[2][6];
        for (int c = 0; c < 6; c++) {
            Ji[0][c] = a00 * Di[0][c] + a02 * Di[2][c];
            Ji[1][c] = a11 * Di[1][c] + a12 * Di[2][c];
            Jj[0][c] = a00 * Dj[0][c] + a02 * Dj[2][c];
            Jj[1][c] = a11 * Dj[1][c] + a12 * Dj[2][c];
        }
        const float Jd0 = a00 * tij[0] + a02 * tij[2], Jd1 = a11 * tij[1] + a12 * tij[2];
        const bool fi = i >= b.n_fixed, fj = j >= b.n_fixed;
        int k = 0;
        for (int a = 0; a < 6; a++)
            for (int c = a; c < 6; c++) v[k++] = fi ? w0 * Ji[0][a] * Ji[0][c] + w1 * Ji[1][a] * Ji[1][c] : 0.f;
        for (int a = 0; a < 6; a++)
            for (int c = 0; c < 6; c++) v[k++] = (fi && fj) ? w0 * Ji[0][a] * Jj[0][c] + w1 * Ji[1][a] * Jj[1][c] : 0.f;
        for (int a = 0; a < 6; a++)
            for (int c = a; c < 6; c++) v[k++] = fj ? w0 * Jj[0][a] * Jj[0][c] + w1 * Jj[1][a] * Jj[1][c] : 0.f;
        for (int a = 0; a < 6; a++) v[k++] = fi ? w0 * Ji[0][a] * r0 + w1 * Ji[1][a] * r1 : 0.f;
        for (int a = 0; a < 6; a++) v[k++] = fj ? w0 * Jj[0][a] * r0 + w1 * Jj[1][a] * r1 : 0.f;
        v[k] = w0 * r0 * r0 + w1 * r1 * r1;
        float* Eo = b.Eb + ((size_t)e * b.P + q) * 12;
        for (int a = 0; a < 6; a++) {
            Eo[a] = fi ? w0 * Ji[0][a] * Jd0 + w1 * Ji[1][a] * Jd1 : 0.f;
            Eo[6 + a] = fj ? w0 * Jj[0][a] * Jd0 + w1 * Jj[1][a] * Jd1 : 0.f;
        }
        atomicAdd(b.C + (size_t)i * b.P + q, w0 * Jd0 * Jd0 + w1 * Jd1 * Jd1);
        atomicAdd(b.gd + (size_t)i * b.P + q, w0 * Jd0 * r0 + w1 * Jd1 * r1);
    }
    const float tot = block_sum_vals(v, s_part);
    const int t = threadIdx.x;
    if (t < kTermVals) {
        const int bi = 6 * (i - b.n_fixed), bj = 6 * (j - b.n_fixed);
        if (t < 21) {
            if (i >= b.n_fixed) {
                int a = 0, c = t, rem = t;          // t -> (a, c), c >= a
                while (rem >= 6 - a) { rem -= 6 - a; a++; }
                c = a + rem;
                atomicAdd(b.S + (size_t)(bi + a) * b.n + bi + c, tot);
                if (c != a) atomicAdd(b.S + (size_t)(bi + c) * b.n + bi + a, tot);
            }
        } else if (t < 57) {
            if (i >= b.n_fixed && j >= b.n_fixed) {
                const int a = (t - 21) / 6, c = (t - 21) % 6;
                atomicAdd(b.S + (size_t)(bi + a) * b.n + bj + c, tot);
                atomicAdd(b.S + (size_t)(bj + c) * b.n + bi + a, tot);
            }
        } else if (t < 78) {
            if (j >= b.n_fixed) {
                int a = 0, rem = t - 57;
                while (rem >= 6 - a) { rem -= 6 - a; a++; }
                const int c = a + rem;
                atomicAdd(b.S + (size_t)(bj + a) * b.n + bj + c, tot);
                if (c != a) atomicAdd(b.S + (size_t)(bj + c) * b.n + bj + a, tot);
            }
        } else if (t < 84) {
            if (i >= b.n_fixed) atomicAdd(b.rhs + bi + (t - 78), -tot);
        } else if (t < 90) {
            if (j >= b.n_fixed) atomicAdd(b.rhs + bj + (t - 84), -tot);
        } else {
            atomicAdd(b.cost, tot);
        }
    }
}

// Levenberg-Marquardt damping of the pose block (before the elimination, so that
// it scales with diag(B) as in the full system).
__global__ void k_ba_damp(BaDev b, float lambda, float eps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < b.n) b.S[(size_t)k * b.n + k] = (1.0f + lambda) * b.S[(size_t)k * b.n + k] + eps;
}

// One CTA per ordered edge pair (e1, e2) with the same source keyframe.
constexpr int kSchurThreads = 160;      // 144 products + spare lanes for the right-hand side
constexpr int kSchurTile = 64;

__global__ void __launch_bounds__(kSchurThreads) k_ba_schur(BaDev b, float lambda, float eps) {
    const int e1 = blockIdx.x, e2 = blockIdx.y;
    const int i = b.ii[e1];
    if (i != b.ii[e2] || !edge_ok(b, i, b.jj[e1]) || !edge_ok(b, i, b.jj[e2])) return;
    __shared__ float s1[kSchurTile][12], s2[kSchurTile][12], sw[kSchurTile], sg[kSchurTile];
    const int t = threadIdx.x;
    const int a = t / 12, c = t % 12;       // product (a, c) of E(e1) E(e2)^T for t < 144
    float acc = 0.f, racc = 0.f;            // racc: (E(e1) C'^-1 g_d)[t - 144] for e1 == e2
    for (int p0 = 0; p0 < b.P; p0 += kSchurTile) {
        const int np = min(kSchurTile, b.P - p0);
        for (int k = t; k < np * 12; k += kSchurThreads) {
            const int pp = k / 12, cc = k % 12;
            s1[pp][cc] = b.Eb[((size_t)e1 * b.P + p0 + pp) * 12 + cc];
            s2[pp][cc] = b.Eb[((size_t)e2 * b.P + p0 + pp) * 12 + cc];
        }
        for (int k = t; k < np; k += kSchurThreads) {
            const float Cp = (1.0f + lambda) * b.C[(size_t)i * b.P + p0 + k] + eps;
            sw[k] = 1.0f / Cp;
            sg[k] = b.gd[(size_t)i * b.P + p0 + k];
        }
        __syncthreads();
        if (t < 144)
            for (int pp = 0; pp < np; pp++) acc += sw[pp] * s1[pp][a] * s2[pp][c];
        else if (t < 156 && e1 == e2)
            for (int pp = 0; pp < np; pp++) racc += sw[pp] * sg[pp] * s1[pp][t - 144];
        __syncthreads();
    }
    const int ji = b.jj[e1], jk = b.jj[e2];
    // slots 0..5: source pose i, 6..11: target pose of the edge
    if (t < 144) {
        const int pa = a < 6 ? i : ji, pc = c < 6 ? i : jk;
        if (pa >= b.n_fixed && pc >= b.n_fixed)
            atomicAdd(b.S + (size_t)(6 * (pa - b.n_fixed) + a % 6) * b.n + 6 * (pc - b.n_fixed) + c % 6, -acc);
    } else if (t < 156 && e1 == e2) {
        const int s = t - 144, pa = s < 6 ? i : ji;
        if (pa >= b.n_fixed) atomicAdd(b.rhs + 6 * (pa - b.n_fixed) + s % 6, racc);
    }
}

// Dense Cholesky solve S x = rhs of the reduced system, one CTA, in shared memory.
constexpr int kSolveThreads = 256;

__global__ void __launch_bounds__(kSolveThreads) k_ba_solve(BaDev b) {
    extern __shared__ float sm[];
    const int n = b.n, t = threadIdx.x;
    float* A = sm;                       // [n][n]
    float* x = sm + n * n;               // [n]
    for (int k = t; k < n * n; k += kSolveThreads) A[k] = b.S[k];
    for (int k = t; k < n; k += kSolveThreads) x[k] = b.rhs[k];
    __syncthreads();
    __shared__ int s_bad;
    if (t == 0) s_bad = 0;
    __syncthreads();
    // right-looking Cholesky, lower triangle
    for (int k = 0; k < n; k++) {
        if (t == 0) {
            const float dkk = A[k * n + k];
            if (!(dkk > 0.f)) s_bad = 1;
            A[k * n + k] = sqrtf(fmaxf(dkk, 1e-30f));
        }
        __syncthreads();
        const float lkk = A[k * n + k];
        for (int r = k + 1 + t; r < n; r += kSolveThreads) A[r * n + k] /= lkk;
        __syncthreads();
        for (int idx = t; idx < (n - k - 1) * (n - k - 1); idx += kSolveThreads) {
            const int r = k + 1 + idx / (n - k - 1), c = k + 1 + idx % (n - k - 1);
            if (c <= r) A[r * n + c] -= A[r * n + k] * A[c * n + k];
        }
        __syncthreads();
    }
    // forward (L y = rhs) and backward (L^T x = y) substitution, one thread per row step
    for (int k = 0; k < n; k++) {
        if (t == 0) x[k] /= A[k * n + k];
        __syncthreads();
        for (int r = k + 1 + t; r < n; r += kSolveThreads) x[r] -= A[r * n + k] * x[k];
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; k--) {
        if (t == 0) x[k] /= A[k * n + k];
        __syncthreads();
        for (int r = t; r < k; r += kSolveThreads) x[r] -= A[k * n + r] * x[k];
        __syncthreads();
    }
    for (int k = t; k < n; k += kSolveThreads) b.dxi[k] = x[k];
    if (t == 0 && s_bad) atomicCAS(b.status, 0, GS_ERR_NUMERIC);
}

__device__ __forceinline__ float pose_dxi(const BaDev& b, int k, int c) {
    return k >= b.n_fixed ? b.dxi[6 * (k - b.n_fixed) + c] : 0.f;
}

// dd_p = C'_p^-1 (-g_d,p - sum_e E(e, p) . [dxi_i, dxi_j]) for every pixel of every
// keyframe; then the poses T_k <- Exp(dxi_k) T_k (rotation exact, translation first order).
__global__ void k_ba_update(BaDev b, float lambda, float eps) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (q < b.P) {
        const float Cp = (1.0f + lambda) * b.C[(size_t)i * b.P + q] + eps;
        float s = -b.gd[(size_t)i * b.P + q];
        for (int e = 0; e < b.E; e++) {
            if (b.ii[e] != i) continue;
            const int j = b.jj[e];
            if (j < 0 || j >= b.K) continue;
            const float* Eo = b.Eb + ((size_t)e * b.P + q) * 12;
            for (int c = 0; c < 6; c++) s -= Eo[c] * pose_dxi(b, i, c) + Eo[6 + c] * pose_dxi(b, j, c);
        }
        // a keyframe that is no edge's source keeps its inverse depths (C = 0 there)
        if (b.C[(size_t)i * b.P + q] > 0.f) b.disp[(size_t)i * b.P + q] += s / Cp;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && i >= b.n_fixed) {
        float rho[3], phi[3];
        for (int c = 0; c < 3; c++) { rho[c] = pose_dxi(b, i, c); phi[c] = pose_dxi(b, i, 3 + c); }
        const float th = sqrtf(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
        const float A = th > 1e-8f ? sinf(th) / th : 1.0f, Bc = th > 1e-8f ? (1.0f - cosf(th)) / (th * th) : 0.5f;
        const float Kx[9] = {0.f, -phi[2], phi[1], phi[2], 0.f, -phi[0], -phi[1], phi[0], 0.f};
        float Rp[9];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                float kk = 0.f;
                for (int m = 0; m < 3; m++) kk += Kx[3 * r + m] * Kx[3 * m + c];
                Rp[3 * r + c] = (r == c ? 1.f : 0.f) + A * Kx[3 * r + c] + Bc * kk;
            }
        // no CTA of this kernel reads the poses (only dxi), so keyframe i's pose can
        // be rewritten here by one thread
        float* P = b.poses + 12 * i;
        float R[9], tt[3];
        for (int m = 0; m < 9; m++) R[m] = P[m];
        for (int m = 0; m < 3; m++) tt[m] = P[9 + m];
        for (int r = 0; r < 3; r++) {
            for (int c = 0; c < 3; c++) P[3 * r + c] = Rp[3 * r] * R[c] + Rp[3 * r + 1] * R[3 + c] + Rp[3 * r + 2] * R[6 + c];
            P[9 + r] = Rp[3 * r] * tt[0] + Rp[3 * r + 1] * tt[1] + Rp[3 * r + 2] * tt[2] + rho[r];
        }
    }
}

}  // namespace

size_t ba_workspace(int K, int E, int P, int n) {
    return align_up(sizeof(float) * (size_t)E * P * 12, 256) + 2 * align_up(sizeof(float) * (size_t)K * P, 256) +
           align_up(sizeof(float) * (size_t)n * n, 256) + 2 * align_up(sizeof(float) * (size_t)(n + 1), 256) +
           align_up(sizeof(float), 256);
}

cudaError_t launch_ba_step(const gs_ba_problem& pr, float lambda, float eps, float* cost, void* ws,
                           cudaStream_t s) {
    BaDev b;
    b.poses = pr.poses; b.disp = pr.disp; b.targets = pr.targets; b.weights = pr.weights;
    b.ii = pr.ii; b.jj = pr.jj;
    b.K = pr.n_keyframes; b.E = pr.n_edges; b.h = pr.height; b.w = pr.width; b.P = pr.height * pr.width;
    b.n_fixed = pr.n_fixed; b.n = 6 * (pr.n_keyframes - pr.n_fixed);
    b.fx = pr.fx; b.fy = pr.fy; b.cx = pr.cx; b.cy = pr.cy;
    char* p = static_cast<char*>(ws);
    b.Eb = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.E * b.P * 12, 256);
    b.C = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.K * b.P, 256);
    b.gd = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.K * b.P, 256);
    b.S = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.n * b.n, 256);
    b.rhs = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)(b.n + 1), 256);
    b.dxi = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)(b.n + 1), 256);
    b.cost = cost;
    b.status = pr.status;
    // zero the accumulators (C, g_d, S, rhs are contiguous after Eb)
    const size_t zero_bytes = 2 * align_up(sizeof(float) * (size_t)b.K * b.P, 256) +
                              align_up(sizeof(float) * (size_t)b.n * b.n, 256) +
                              align_up(sizeof(float) * (size_t)(b.n + 1), 256);
    cudaError_t e = cudaMemsetAsync(b.C, 0, zero_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cost, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (b.E > 0) {
        k_ba_terms<<<dim3((unsigned)ceil_div(b.P, kTermThreads), (unsigned)b.E), kTermThreads, 0, s>>>(b);
        if (b.n > 0) {
            k_ba_damp<<<(unsigned)ceil_div(b.n, 256), 256, 0, s>>>(b, lambda, eps);
            k_ba_schur<<<dim3((unsigned)b.E, (unsigned)b.E), kSchurThreads, 0, s>>>(b, lambda, eps);
            const size_t smem = sizeof(float) * ((size_t)b.n * b.n + b.n);
            e = cudaFuncSetAttribute(k_ba_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_ba_solve<<<1, kSolveThreads, smem, s>>>(b);
        }
        k_ba_update<<<dim3((unsigned)ceil_div(b.P, 256), (unsigned)b.K), 256, 0, s>>>(b, lambda, eps);
    }
    return cudaGetLastError();
}

}  // namespace gs
