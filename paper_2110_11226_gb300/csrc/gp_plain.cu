// gp_plain.cu -- the plain evaluator: one launch per program, the shape of
// the paper's execution kernel (Sec. III-C3): one row per thread, 256
// threads per block, every thread of the grid on the same program, the
// prefix list scanned in reverse straight from global memory, and a
// fixed-size stack whose push and pop are unrolled loops over all 20 slots
// so that the slots stay in registers (Sec. III-B, III-D1).  The loss is
// fused and each block writes one partial sum; the shared finalize pass
// adds them in FP64.  It is the comparison point for the batched evaluator.
#include "gp_internal.cuh"
#include "gp_math.cuh"

namespace gpk {

namespace {

__device__ __forceinline__ float p_loss(int metric, float p, float y) {
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

struct Stack {
    float v[GP_MAX_STACK];
    int sp = 0;
    __device__ __forceinline__ void push(float x) {
#pragma unroll
        for (int i = 0; i < GP_MAX_STACK; ++i)
            if (i == sp) v[i] = x;
        ++sp;
    }
    __device__ __forceinline__ float pop() {
        float x = 0.0f;
        --sp;
#pragma unroll
        for (int i = 0; i < GP_MAX_STACK; ++i)
            if (i == sp) x = v[i];
        return x;
    }
};

}  // namespace

__global__ void __launch_bounds__(256) plain_kernel(PlainArgs a, int p) {
    __shared__ float red[8];
    const ProgMeta m = a.meta[p];
    const int64_t row = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const bool valid = row < a.n_rows;
    float e = 0.0f;
    if (m.status == GP_PROG_OK) {
        const int off = a.offsets[p];
        const int len = a.offsets[p + 1] - off;
        const gp_node *prog = a.progs + off;
        const int64_t r = valid ? row : 0;
        Stack st;
        for (int j = len - 1; j >= 0; --j) {
            const gp_node nd = prog[j];
            const int op = nd.op;
            if (op == GP_CONST) {
                st.push(nd.c);
            } else if (op == GP_VAR) {
                st.push(valid ? __ldg(a.X + (int64_t)nd.feat * a.ld + r) : 0.0f);
            } else if (op >= GP_SQRT && op <= GP_COSH) {
                const float x = st.pop();
                float z;
                if (op == GP_SQRT) z = __fsqrt_rn(fabsf(x));
                else if (op == GP_LOG) z = fabsf(x) < kThr ? 0.0f : logf(fabsf(x));
                else if (op == GP_EXP) z = expf(x);
                else if (op == GP_SIN) z = sinf(x);
                else if (op == GP_COS) z = cosf(x);
                else if (op == GP_TAN) z = tanf(x);
                else if (op == GP_ABS) z = fabsf(x);
                else if (op == GP_NEG) z = -x;
                else if (op == GP_INV) z = fabsf(x) < kThr ? 0.0f : __frcp_rn(x);
                else if (op == GP_SQ) z = f_sq(x);
                else if (op == GP_CUBE) z = f_cube(x);
                else if (op == GP_CBRT) z = f_cbrt(x);
                else if (op == GP_TANH) z = f_tanh(x);
                else if (op == GP_ATAN) z = f_atan(x);
                else if (op == GP_SINH) z = f_sinh(x);
                else z = f_cosh(x);
                st.push(z);
            } else {
                const float l = st.pop();
                const float rr = st.pop();
                float z;
                if (op == GP_ADD) z = __fadd_rn(l, rr);
                else if (op == GP_SUB) z = __fsub_rn(l, rr);
                else if (op == GP_MUL) z = __fmul_rn(l, rr);
                else if (op == GP_DIV) z = fabsf(rr) < kThr ? 1.0f : __fdiv_rn(l, rr);
                else if (op == GP_MAX) z = f_max(l, rr);
                else z = f_min(l, rr);
                st.push(z);
            }
        }
        const float pred = st.pop();
        if (valid) {
            e = p_loss(a.metric, pred, __ldg(a.y + r));
            if (a.w) e = __fmul_rn(__ldg(a.w + r), e);
        }
    } else {
        e = __int_as_float(0x7fc00000);
    }
    // fixed-order block reduction: butterfly per warp, then warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = __fadd_rn(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < 8; ++i) s = __fadd_rn(s, red[i]);
        a.part[(size_t)p * a.n_blocks + blockIdx.x] = s;
    }
}

cudaError_t launch_plain(const PlainArgs &a, int p, cudaStream_t st) {
    plain_kernel<<<a.n_blocks, 256, 0, st>>>(a, p);
    return cudaGetLastError();
}

}  // namespace gpk
