// gp_grad.cu -- gradients of fitness with respect to the ephemeral
// constants (reverse mode), and one Adam step on the constants.  Neither
// has a counterpart in the paper; they serve constant tuning between
// generations.
//
// Per row, the forward values of all nodes are recomputed (children have
// larger prefix positions, so a reverse sweep over the list computes each
// node from already computed children with the same FP32 operations as the
// stack evaluator) and kept in per-thread local memory; nothing of size
// programs x rows x nodes is ever stored.  The adjoint sweep then runs in
// prefix order, parents before children: the root gets w * dl/dp and every
// function hands its children their share; a constant adds its node's
// adjoint into its slot.  Per-thread sums are Kahan-compensated FP32, warp
// sums fixed-order, cross-chunk sums FP64 (gp_reduce.cu).
#include "gp_internal.cuh"
#include "gp_math.cuh"

namespace gpk {

namespace {

constexpr int kGradBlock = 128;

__device__ __forceinline__ void kahan(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = isfinite(t) ? __fsub_rn(__fsub_rn(t, s), y) : 0.0f;
    s = t;
}

__device__ __forceinline__ float sgnf(float x) {
    return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f);
}

__device__ __forceinline__ float g_loss(int metric, float p, float y) {
    if (metric == GP_MAE) return fabsf(__fsub_rn(p, y));
    if (metric == GP_LOGLOSS) {
        const float ap = fabsf(p);
        const float c = (p >= 0.0f) ? __fsub_rn(1.0f, y) : y;
        const float lin = (c == 0.0f) ? 0.0f : __fmul_rn(c, ap);
        return __fadd_rn(lin, log1pf(expf(-ap)));
    }
    const float d = __fsub_rn(p, y);
    return __fmul_rn(d, d);
}

__device__ __forceinline__ float g_dloss(int metric, float p, float y) {
    if (metric == GP_MAE) return sgnf(__fsub_rn(p, y));
    if (metric == GP_LOGLOSS) {
        float s;
        if (p >= 0.0f) {
            s = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-p)));
        } else {
            const float e = expf(p);
            s = __fdiv_rn(e, __fadd_rn(1.0f, e));
        }
        return __fsub_rn(s, y);
    }
    return __fmul_rn(2.0f, __fsub_rn(p, y));
}

__device__ __forceinline__ float g_f1(int op, float a) {
    switch (op) {
    case GP_SQRT: return __fsqrt_rn(fabsf(a));
    case GP_LOG: return fabsf(a) < kThr ? 0.0f : logf(fabsf(a));
    case GP_EXP: return expf(a);
    case GP_SIN: return sinf(a);
    case GP_COS: return cosf(a);
    case GP_TAN: return tanf(a);
    case GP_ABS: return fabsf(a);
    case GP_NEG: return -a;
    case GP_INV: return fabsf(a) < kThr ? 0.0f : __frcp_rn(a);
    case GP_SQ: return f_sq(a);
    case GP_CUBE: return f_cube(a);
    case GP_CBRT: return f_cbrt(a);
    case GP_TANH: return f_tanh(a);
    case GP_ATAN: return f_atan(a);
    case GP_SINH: return f_sinh(a);
    default: return f_cosh(a);
    }
}

__device__ __forceinline__ float g_f2(int op, float l, float r) {
    switch (op) {
    case GP_ADD: return __fadd_rn(l, r);
    case GP_SUB: return __fsub_rn(l, r);
    case GP_MUL: return __fmul_rn(l, r);
    case GP_DIV: return fabsf(r) < kThr ? 1.0f : __fdiv_rn(l, r);
    case GP_MAX: return f_max(l, r);
    default: return f_min(l, r);
    }
}

__device__ __forceinline__ bool is_unary(int op) { return op >= GP_SQRT && op <= GP_COSH; }

}  // namespace

__global__ void __launch_bounds__(kGradBlock) grad_kernel(GradArgs a) {
    __shared__ gp_node s_nodes[kGradBlock / 32][kCodeStride];
    __shared__ uint8_t s_rc[kGradBlock / 32][kCodeStride];
    __shared__ int8_t s_ks[kGradBlock / 32][kCodeStride];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    gp_node *nodes = s_nodes[wi];
    uint8_t *rc = s_rc[wi];
    int8_t *ks = s_ks[wi];
    const unsigned long long total =
        (unsigned long long)a.n_progs * (unsigned long long)a.n_chunks;
    float val[GP_MAX_LEN], adj[GP_MAX_LEN];

    for (unsigned long long it = 0; it <= total; ++it) {
        if (it == total) {
            if (lane == 0) atomicOr(a.dev_status, GP_DEV_QUEUE_CAP);
            break;
        }
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int chunk = (int)(item / (unsigned long long)a.n_progs);
        const int rank = (int)(item - (unsigned long long)chunk * a.n_progs);
        const int p = a.order[rank];
        const ProgMeta m = a.meta[p];
        float *gp = a.gpart + ((size_t)p * a.n_chunks + chunk) * GP_MAX_CONSTS;
        if (m.status != GP_PROG_OK || m.n_consts > GP_MAX_CONSTS) {
            if (lane == 0) {
                a.part[(size_t)p * a.n_chunks + chunk] = __int_as_float(0x7fc00000);
                for (int k = 0; k < GP_MAX_CONSTS; ++k) gp[k] = __int_as_float(0x7fc00000);
                if (m.n_consts > GP_MAX_CONSTS) atomicOr(a.dev_status, GP_DEV_TOO_MANY_CONSTS);
            }
            continue;
        }
        const int off = a.offsets[p];
        const int len = a.offsets[p + 1] - off;
        __syncwarp();
        for (int i = lane; i < len; i += 32) {
            nodes[i] = a.progs[off + i];
            rc[i] = a.rchild[(size_t)p * kCodeStride + i];
            ks[i] = a.kslot[(size_t)p * kCodeStride + i];
        }
        __syncwarp();

        const int64_t rb = (int64_t)chunk * a.chunk_rows;
        const int64_t re = min(a.n_rows, rb + a.chunk_rows);
        float gs[GP_MAX_CONSTS], gc[GP_MAX_CONSTS];
#pragma unroll
        for (int k = 0; k < GP_MAX_CONSTS; ++k) gs[k] = gc[k] = 0.0f;
        float ls = 0.0f, lc = 0.0f;
        for (int64_t r = rb + lane; r < re; r += 32) {
            // forward: children before parents
            for (int j = len - 1; j >= 0; --j) {
                const gp_node nd = nodes[j];
                float v;
                if (nd.op == GP_CONST) v = nd.c;
                else if (nd.op == GP_VAR) v = __ldg(a.X + (int64_t)nd.feat * a.ld + r);
                else if (is_unary(nd.op)) v = g_f1(nd.op, val[j + 1]);
                else v = g_f2(nd.op, val[j + 1], val[j + rc[j]]);
                val[j] = v;
            }
            const float pr = val[0];
            const float yv = __ldg(a.y + r);
            const float wv = a.w ? __ldg(a.w + r) : 1.0f;
            kahan(ls, lc, __fmul_rn(wv, g_loss(a.metric, pr, yv)));
            // adjoint: parents before children
            adj[0] = __fmul_rn(wv, g_dloss(a.metric, pr, yv));
            for (int j = 0; j < len; ++j) {
                const gp_node nd = nodes[j];
                const float aj = adj[j];
                if (nd.op == GP_CONST) {
                    const int k = ks[j];
#pragma unroll
                    for (int q = 0; q < GP_MAX_CONSTS; ++q)
                        if (q == k) kahan(gs[q], gc[q], aj);
                    continue;
                }
                if (nd.op == GP_VAR) continue;
                const float u = val[j + 1];
                if (is_unary(nd.op)) {
                    float du;
                    switch (nd.op) {
                    case GP_SQRT: du = (u == 0.0f) ? 0.0f : __fdiv_rn(sgnf(u), __fmul_rn(2.0f, val[j])); break;
                    case GP_LOG: du = fabsf(u) < kThr ? 0.0f : __frcp_rn(u); break;
                    case GP_EXP: du = val[j]; break;
                    case GP_SIN: du = cosf(u); break;
                    case GP_COS: du = -sinf(u); break;
                    case GP_TAN: du = __fadd_rn(1.0f, __fmul_rn(val[j], val[j])); break;
                    case GP_ABS: du = sgnf(u); break;
                    case GP_NEG: du = -1.0f; break;
                    case GP_INV: du = fabsf(u) < kThr ? 0.0f : -__fmul_rn(val[j], val[j]); break;
                    case GP_SQ: du = __fmul_rn(2.0f, u); break;
                    case GP_CUBE: du = __fmul_rn(3.0f, __fmul_rn(u, u)); break;
                    case GP_CBRT:
                        du = (u == 0.0f) ? 0.0f : __frcp_rn(__fmul_rn(3.0f, __fmul_rn(val[j], val[j])));
                        break;
                    case GP_TANH: du = __fsub_rn(1.0f, __fmul_rn(val[j], val[j])); break;
                    case GP_ATAN: du = __frcp_rn(__fadd_rn(1.0f, __fmul_rn(u, u))); break;
                    case GP_SINH: du = coshf(u); break;
                    default: du = sinhf(u); break;  // GP_COSH
                    }
                    adj[j + 1] = __fmul_rn(aj, du);
                } else {
                    const float v = val[j + rc[j]];
                    float du, dv;
                    switch (nd.op) {
                    case GP_ADD: du = 1.0f; dv = 1.0f; break;
                    case GP_SUB: du = 1.0f; dv = -1.0f; break;
                    case GP_MUL: du = v; dv = u; break;
                    case GP_DIV:
                        if (fabsf(v) < kThr) { du = 0.0f; dv = 0.0f; }
                        else { du = __frcp_rn(v); dv = -__fdiv_rn(val[j], v); }
                        break;
                    case GP_MAX:
                        du = (u > v || u != u) ? 1.0f : 0.0f;
                        dv = __fsub_rn(1.0f, du);
                        break;
                    default:  // GP_MIN
                        du = (u < v || u != u) ? 1.0f : 0.0f;
                        dv = __fsub_rn(1.0f, du);
                        break;
                    }
                    adj[j + 1] = __fmul_rn(aj, du);
                    adj[j + rc[j]] = __fmul_rn(aj, dv);
                }
            }
        }
        float lv = __fsub_rn(ls, lc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lv = __fadd_rn(lv, __shfl_xor_sync(0xffffffffu, lv, o));
        float gv[GP_MAX_CONSTS];
#pragma unroll
        for (int k = 0; k < GP_MAX_CONSTS; ++k) {
            gv[k] = __fsub_rn(gs[k], gc[k]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gv[k] = __fadd_rn(gv[k], __shfl_xor_sync(0xffffffffu, gv[k], o));
        }
        if (lane == 0) {
            a.part[(size_t)p * a.n_chunks + chunk] = lv;
#pragma unroll
            for (int k = 0; k < GP_MAX_CONSTS; ++k) gp[k] = gv[k];
        }
    }
}

// Latency-bound (per node a dependent chain through the per-thread value
// and adjoint arrays in local memory), so the launch fills every SM: at 16
// warps per SM a Pagie-1 1M x 2048 gradient pass took 245 ms, at 32 warps
// 159 ms, at 8 warps 410 ms.
int info_grad() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grad_kernel, kGradBlock, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_grad(const GradArgs &a, int grid, int block, cudaStream_t st) {
    (void)block;
    grad_kernel<<<grid, kGradBlock, 0, st>>>(a);
    return cudaGetLastError();
}

// Adam: one thread per program walks its prefix list; the k-th CONST node
// takes slot k of grad / m / v.
__global__ void __launch_bounds__(128) adam_kernel(AdamArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_progs) return;
    const int off = a.offsets[p];
    const int len = a.offsets[p + 1] - off;
    if (len < 1 || len > GP_MAX_LEN) return;
    const float b1t = 1.0f - powf(a.beta1, (float)a.step);
    const float b2t = 1.0f - powf(a.beta2, (float)a.step);
    int k = 0;
    for (int j = 0; j < len && k < GP_MAX_CONSTS; ++j) {
        gp_node *nd = a.progs + off + j;
        if (nd->op != GP_CONST) continue;
        const size_t i = (size_t)p * GP_MAX_CONSTS + k;
        const float g = a.grad[i];
        if (isfinite(g)) {
            const float mi = __fadd_rn(__fmul_rn(a.beta1, a.m[i]), __fmul_rn(1.0f - a.beta1, g));
            const float vi = __fadd_rn(__fmul_rn(a.beta2, a.v[i]),
                                       __fmul_rn(1.0f - a.beta2, __fmul_rn(g, g)));
            a.m[i] = mi;
            a.v[i] = vi;
            const float mh = __fdiv_rn(mi, b1t);
            const float vh = __fdiv_rn(vi, b2t);
            const float stp = __fdiv_rn(__fmul_rn(a.lr, mh), __fadd_rn(__fsqrt_rn(vh), a.eps));
            nd->c = __fsub_rn(nd->c, stp);
        }
        ++k;
    }
}

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st) {
    if (a.n_progs <= 0) return cudaSuccess;
    adam_kernel<<<(a.n_progs + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// One thread per program: the k-th CONST node in prefix order is slot k.
__global__ void __launch_bounds__(128) consts_kernel(gp_node *progs, const int32_t *offsets,
                                                     int n_progs, float *consts, bool to_nodes) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_progs) return;
    const int off = offsets[p];
    const int len = offsets[p + 1] - off;
    float *row = consts + (size_t)p * GP_MAX_CONSTS;
    int k = 0;
    if (len >= 1 && len <= GP_MAX_LEN) {
        for (int j = 0; j < len && k < GP_MAX_CONSTS; ++j) {
            gp_node *nd = progs + off + j;
            if (nd->op != GP_CONST) continue;
            if (to_nodes) nd->c = row[k];
            else row[k] = nd->c;
            ++k;
        }
    }
    if (!to_nodes)
        for (; k < GP_MAX_CONSTS; ++k) row[k] = 0.0f;
}

cudaError_t launch_consts(gp_node *progs, const int32_t *offsets, int n_progs, float *consts,
                          bool to_nodes, cudaStream_t st) {
    if (n_progs <= 0) return cudaSuccess;
    consts_kernel<<<(n_progs + 127) / 128, 128, 0, st>>>(progs, offsets, n_progs, consts, to_nodes);
    return cudaGetLastError();
}

}  // namespace gpk
