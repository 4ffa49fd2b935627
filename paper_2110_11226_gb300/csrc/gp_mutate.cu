// gp_mutate.cu -- the mutation step on the device: the next population is
// built from tournament winners without leaving the GPU (the paper mutates
// on the CPU and copies every program back, Sec. III-C2 and III-D2, and
// names avoiding those transfers as future work, Sec. V).
//
// Three launches: one thread per offspring draws its kind and builds the
// child in its own 256-node scratch slot (Sec. II-A crossover, subtree,
// hoist and point mutation, reproduction; the hoisted crossover of
// Sec. III-C2 keeps the child within 20 stack slots and 255 nodes); one
// block turns the children's lengths into offsets; one warp per child
// copies it into the packed output.  Every random word comes from the
// offspring's own Philox4x32-10 stream, word k = Philox(counter = (k/4, t,
// offset lo32, offset hi32), key = seed)[k%4], so the output depends on
// nothing but the inputs.
#include "gp_internal.cuh"

namespace gpk {
namespace {

constexpr int kSlot = 256;  // scratch nodes per offspring

struct Stream {
    uint2 key;
    uint32_t t, c2, c3, k;
    uint4 r;
};

__device__ __forceinline__ uint32_t next_word(Stream &s) {
    if ((s.k & 3) == 0) s.r = philox4x32_10(make_uint4(s.k >> 2, s.t, s.c2, s.c3), s.key);
    const uint32_t w = (s.k & 3) == 0 ? s.r.x : (s.k & 3) == 1 ? s.r.y : (s.k & 3) == 2 ? s.r.z : s.r.w;
    s.k += 1;
    return w;
}

// an index in [0, n) from one word
__device__ __forceinline__ int pick(Stream &s, int n) {
    return (int)(((uint64_t)next_word(s) * (uint64_t)n) >> 32);
}

__device__ __forceinline__ int arity_of(int op) {
    if (op == GP_CONST || op == GP_VAR) return 0;
    if ((op >= GP_ADD && op <= GP_DIV) || op == GP_MAX || op == GP_MIN) return 2;
    if (op >= GP_SQRT && op <= GP_COSH) return 1;
    return -1;
}

// the reverse scan of Sec. III-A: validity of a prefix list
__device__ bool valid_program(const gp_node *p, int len, int n_feat) {
    if (len < 1 || len > GP_MAX_LEN) return false;
    int sp = 0, hw = 0;
    for (int j = len - 1; j >= 0; --j) {
        const int a = arity_of(p[j].op);
        if (a < 0) return false;
        if (p[j].op == GP_VAR && (p[j].feat < 0 || p[j].feat >= n_feat)) return false;
        if (sp < a) return false;
        sp += 1 - a;
        hw = max(hw, sp);
    }
    return sp == 1 && hw <= GP_MAX_STACK;
}

// nodes of the subtree rooted at node i
__device__ int subtree_size(const gp_node *p, int len, int i) {
    int need = 1;
    for (int m = i; m < len; ++m) {
        need += arity_of(p[m].op) - 1;
        if (need == 0) return m - i + 1;
    }
    return len - i;  // unreachable for a valid program
}

// variable f for f < n_feat, else a constant (w >> 8) * 2^-23 - 1 from the
// next word (exact in float, uniform on [-1, 1))
__device__ gp_node new_terminal(Stream &s, int n_feat) {
    gp_node nd;
    nd.op = GP_CONST;
    nd.feat = 0;
    nd.c = 0.0f;
    const int f = pick(s, n_feat + 1);
    if (f < n_feat) {
        nd.op = GP_VAR;
        nd.feat = (int16_t)f;
    } else {
        const uint32_t w = next_word(s);
        nd.c = __fsub_rn(__fmul_rn((float)(w >> 8), 0x1p-23f), 1.0f);
    }
    return nd;
}

// a "grow" tree of depth <= limit (<= 6, so <= 127 nodes) in prefix order:
// below the limit a node is a terminal when a word picks one of the 2
// terminal kinds among 2 + n_funcs, else one of the allowed functions
__device__ int grow_tree(Stream &s, const MutArgs &a, gp_node *out) {
    int8_t slot_depth[2 * 64];
    int top = 0, n = 0;
    slot_depth[top++] = 0;
    while (top > 0 && n < 127) {
        const int d = slot_depth[--top];
        const bool terminal = d >= a.subtree_depth || pick(s, a.n_funcs + 2) < 2;
        if (terminal) {
            out[n++] = new_terminal(s, a.n_feat);
        } else {
            gp_node nd;
            nd.op = a.funcs[pick(s, a.n_funcs)];
            nd.feat = 0;
            nd.c = 0.0f;
            out[n++] = nd;
            for (int k = 0; k < arity_of(nd.op); ++k) slot_depth[top++] = (int8_t)(d + 1);
        }
    }
    return n;
}

// Length of the parent with subtree [i, i+si) replaced by donor subtree
// [j, j+sj), or 0 when that child would exceed 255 nodes or 20 stack
// slots; the stack height is scanned over the three pieces in place.
__device__ int splice_len(const gp_node *par, int lp, int i, int si, const gp_node *don, int j,
                          int sj) {
    const int len = i + sj + (lp - i - si);
    if (len > GP_MAX_LEN) return 0;
    int sp = 0, hw = 0;
    for (int m = lp - 1; m >= i + si; --m) {
        sp += 1 - arity_of(par[m].op);
        hw = max(hw, sp);
    }
    for (int m = j + sj - 1; m >= j; --m) {
        sp += 1 - arity_of(don[m].op);
        hw = max(hw, sp);
    }
    for (int m = i - 1; m >= 0; --m) {
        sp += 1 - arity_of(par[m].op);
        hw = max(hw, sp);
    }
    return hw <= GP_MAX_STACK ? len : 0;
}

__device__ void splice_write(const gp_node *par, int lp, int i, int si, const gp_node *don, int j,
                             int sj, gp_node *out) {
    int n = 0;
    for (int m = 0; m < i; ++m) out[n++] = par[m];
    for (int m = j; m < j + sj; ++m) out[n++] = don[m];
    for (int m = i + si; m < lp; ++m) out[n++] = par[m];
}

// the hoisted crossover: while the child does not fit, the donor subtree
// moves to a node drawn among its proper descendants
__device__ int hoisted_splice(Stream &s, const gp_node *par, int lp, int i, const gp_node *don,
                              int ld, int j, gp_node *out) {
    const int si = subtree_size(par, lp, i);
    int sj = subtree_size(don, ld, j);
    for (int guard = 0; guard <= GP_MAX_LEN; ++guard) {
        const int len = splice_len(par, lp, i, si, don, j, sj);
        if (len > 0) {
            splice_write(par, lp, i, si, don, j, sj, out);
            return len;
        }
        if (sj == 1) return 0;  // a terminal always fits a valid parent
        j = j + 1 + pick(s, sj - 1);
        sj = subtree_size(don, ld, j);
    }
    return 0;
}

__global__ void __launch_bounds__(128) mutate_plan_kernel(const MutArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_out) return;
    gp_node *child = a.scratch + (size_t)t * kSlot;
    Stream s;
    s.key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    s.t = (uint32_t)t;
    s.c2 = (uint32_t)a.offset;
    s.c3 = (uint32_t)(a.offset >> 32);
    s.k = 0;
    const uint32_t u = next_word(s);
    int kind = GP_MUT_REPRODUCTION;
    for (int q = 0; q < 4; ++q)
        if ((uint64_t)u < a.thr[q]) {
            kind = q + 1;
            break;
        }
    const int pi = a.parents[2 * t], di = a.parents[2 * t + 1];
    gp_node zero;
    zero.op = GP_CONST;
    zero.feat = 0;
    zero.c = 0.0f;
    if (pi < 0 || pi >= a.n_progs || di < 0 || di >= a.n_progs) {
        atomicOr(a.dev_status, GP_DEV_BAD_PARENT);
        child[0] = zero;
        a.lens[t] = 1;
        if (a.kind) a.kind[t] = GP_MUT_REPRODUCTION;
        return;
    }
    const gp_node *par = a.progs + a.offsets[pi];
    int lp = a.offsets[pi + 1] - a.offsets[pi];
    const gp_node *don = a.progs + a.offsets[di];
    const int ld = a.offsets[di + 1] - a.offsets[di];
    if (!valid_program(par, lp, a.n_feat)) {
        kind = GP_MUT_REPRODUCTION;
        if (lp < 1 || lp > GP_MAX_LEN) {
            child[0] = zero;
            par = child;
            lp = 1;
        }
    }
    if (kind == GP_MUT_CROSSOVER && !valid_program(don, ld, a.n_feat)) kind = GP_MUT_REPRODUCTION;

    int len = 0;
    if (kind == GP_MUT_CROSSOVER) {
        const int i = pick(s, lp);
        const int j = pick(s, ld);
        len = hoisted_splice(s, par, lp, i, don, ld, j, child);
    } else if (kind == GP_MUT_SUBTREE) {
        gp_node tree[128];
        const int lt = grow_tree(s, a, tree);
        const int i = pick(s, lp);
        len = hoisted_splice(s, par, lp, i, tree, lt, 0, child);
    } else if (kind == GP_MUT_HOIST) {
        const int i = pick(s, lp);
        const int si = subtree_size(par, lp, i);
        const int k = si > 1 ? i + 1 + pick(s, si - 1) : i;
        len = splice_len(par, lp, i, si, par, k, subtree_size(par, lp, k));
        if (len > 0) splice_write(par, lp, i, si, par, k, subtree_size(par, lp, k), child);
    } else if (kind == GP_MUT_POINT) {
        for (int m = 0; m < lp; ++m) child[m] = par[m];
        len = lp;
        for (int m = 0; m < lp; ++m) {
            if ((uint64_t)next_word(s) >= a.thr_replace) continue;
            const int ar = arity_of(par[m].op);
            if (ar == 0) {
                child[m] = new_terminal(s, a.n_feat);
            } else {
                const int ns = ar == 1 ? a.n_unary : a.n_binary;
                if (ns > 0) {
                    const int idx = pick(s, ns);
                    child[m].op = ar == 1 ? a.unary[idx] : a.binary[idx];
                    child[m].feat = 0;
                    child[m].c = 0.0f;
                }
            }
        }
    }
    if (len == 0) {  // reproduction, or a splice that could not fit
        if (par != child)
            for (int m = 0; m < lp; ++m) child[m] = par[m];
        len = lp;
        kind = GP_MUT_REPRODUCTION;
    }
    a.lens[t] = len;
    if (a.kind) a.kind[t] = kind;
}

// exclusive scan of the lengths in one block, 1024 at a time with a carry
__global__ void __launch_bounds__(1024) mutate_scan_kernel(const MutArgs a) {
    __shared__ int32_t warp_sum[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < a.n_out; base += 1024) {
        const int t = base + (int)threadIdx.x;
        const int32_t v = t < a.n_out ? a.lens[t] : 0;
        int32_t x = v;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
        if (t < a.n_out) a.out_offsets[t] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.out_offsets[a.n_out] = carry;
}

// one warp per child: scratch slot -> packed output
__global__ void __launch_bounds__(256) mutate_copy_kernel(const MutArgs a) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= a.n_out) return;
    const int len = a.lens[t];
    const gp_node *src = a.scratch + (size_t)t * kSlot;
    gp_node *dst = a.out + a.out_offsets[t];
    for (int m = lane; m < len; m += 32) dst[m] = src[m];
}

}  // namespace

cudaError_t launch_mutate(const MutArgs &a, cudaStream_t st) {
    if (a.n_out <= 0) return cudaSuccess;
    mutate_plan_kernel<<<(a.n_out + 127) / 128, 128, 0, st>>>(a);
    mutate_scan_kernel<<<1, 1024, 0, st>>>(a);
    mutate_copy_kernel<<<(a.n_out * 32 + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gpk
