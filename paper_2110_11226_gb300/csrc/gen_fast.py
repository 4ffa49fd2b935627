"""Write gp_fast.cuh: the evaluator's indexed-branch fast loop in inline PTX.

The loop runs the compiled instruction words of one program (the format of
gp_internal.cuh) over RPT rows per lane, RPT = 4 or 8.  A lane's rows are
held as RPT/2 pairs of 32-bit floats in 64-bit registers, and every
operation that rounds each row on its own -- add, sub, mul and fma -- runs
as one packed instruction per pair (add/sub/mul/fma.rn.f32x2: round to
nearest per element, no flush to zero, so the bits are those of the scalar
instructions).  Divisions, square roots, reciprocals and the selects of
the protected operators run per row.  One word is dispatched by one
indexed branch (brx.idx through a 64-entry table on the low six bits of
the word).

sin, cos, log and exp transcribe the steps and constants of gp_math.cuh
(sincos_fast, log_pos, exp_fast), so the loop and the C++ fallback give the
same bits; the constants are written here as the bit patterns that
gp_math.cuh's static_asserts pin.  Code size matters as much as
instruction count (at 8 rows per lane an unrolled body per operation
overflowed the instruction cache: ncu's no_instruction stall rose to 4 per
issue), so the division forms share one body (the divisor staged in U;
the reversed forms swap the rows into U first), sin and cos share one,
and tan goes to the C++ switch.

Variants: RPT in {4, 8} x DIVS (the division set, square root, reciprocal,
sin, cos, log and exp run here; without DIVS they are handed back) x
XREG (columns 0 and 1 held in registers; without it every column read is
handed back).  A word the loop does not run -- END, the extended
functions, the trigonometric and exponential arguments outside their fast
paths, and whatever DIVS or XREG leave out -- is handed back to the
caller's switch with its constant, the address just past it, and the rows
untouched.

Run: python paper_2110_11226_gb300/csrc/gen_fast.py  (rewrites gp_fast.cuh)
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))

# op codes (gp_internal.cuh); bit 5 of a column-read word picks column 1
OPS = dict(PUSH_X=0, PUSH_C=1, PUSH_X_SP=2, PUSH_C_SP=3, ADD_S=4, SUB_S=5, MUL_S=6, DIV_S=7,
           ADD_X=8, ADD_C=9, SUB_X=10, SUB_C=11, RSUB_X=12, RSUB_C=13, MUL_X=14, MUL_C=15,
           DIV_X=16, DIV_C=17, RDIV_X=18, RDIV_C=19, SQRT=20, LOG=21, EXP=22, SIN=23, COS=24,
           TAN=25, ABS=26, NEG=27, INV=28, END=29, EXT1=30, EXT2=31)
COL1 = 32

# float bit patterns (pinned by static_asserts in gp_math.cuh)
K = dict(inv_pi=0x3EA2F983, magic=0x4B400000, pi_hi=0x40490FDB, pi_mid=0xB3BBBD2E,
         pi_lo=0xA7772CED, q0=0xBE2AAAA6, q1=0x3C088769, q2=0xB94FB7D4, q3=0x362EDC67,
         trig_fast=0x47800000,
         lp0=0xBEFFFFFD, lp1=0x3EAAAB7A, lp2=0xBE80024D, lp3=0x3E4C6960, lp4=0xBE29AE98,
         lp5=0x3E18C293, lp6=0xBE12824F, lp7=0x3DB2E3B9, ln2_hi=0x3F317200, ln2_lo=0x35BFBE8E,
         e1=0x3F800000, e2=0x3EFFFFFE, e3=0x3E2AAA06, e4=0x3D2AAC20, e5=0x3C09371C,
         e6=0x3AB57078, log2e=0x3FB8AA3B, exp_fast=0x42AE0000, one=0x3F800000,
         mhalf=0xBF000000, flt_max=0x7F7FFFFF, half=0x3F000000, mone=0xBF800000,
         inf=0x7F800000, two_m100=0x0D800000, two_126=0x7E800000, two_60=0x5D800000,
         two_m60=0x21800000, exp_inf=0x42B20000, exp_zero=0xC2DC0000)
NEG = 0x80000000


def kf(name, neg=False):
    """a float immediate: 0fXXXXXXXX"""
    return f"0f{(K[name] ^ (NEG if neg else 0)):08X}"


def kp(name, neg=False):
    """a 64-bit immediate holding the constant in both halves"""
    b = K[name] ^ (NEG if neg else 0)
    return f"0x{b:08X}{b:08X}"


class Gen:
    def __init__(self, rpt, divs, xreg, grad=False):
        self.rpt, self.divs, self.xreg, self.grad = rpt, divs, xreg, grad
        self.np = rpt // 2               # pairs per lane
        p = self.np
        self.T = [f"%{1 + i}" for i in range(p)]
        self.HW, self.HC, self.SB, self.NSM1 = f"%{p + 1}", f"%{p + 2}", f"%{p + 3}", f"%{p + 4}"
        self.X = [[f"%{p + 5 + i}" for i in range(p)], [f"%{2 * p + 5 + i}" for i in range(p)]]
        self.THR = f"%{3 * p + 5}"
        # gradient variant: the lane's tangent slot 0 and the tangent slots
        self.DB, self.KT = f"%{3 * p + 6}", f"%{3 * p + 7}"
        self.slot_bytes = (rpt // 4) * 512
        self.lines = []
        # the special-value paths (4 rows per lane only: at 8 the loop's
        # larger code made the evaluator 2.3% slower on Pagie-1 16M x 4096)
        self.special = rpt == 4
        self.nsv = 0          # special-value paths emitted so far
        self.deferred = []    # their blocks, emitted after the bodies

    # -- emission helpers -------------------------------------------------
    def e(self, s):
        self.lines.append(s)

    def label(self, name):
        self.lines.append(f"{name}%=:")

    def nxt(self):
        # the gradient variant returns through ret: 0 = the next word, else
        # the partial-derivative body of the marked word just run
        self.e("brx.idx.uni %%ret, TR%=;" if self.grad else "bra.uni N%=;")

    def unpack(self, i, a, b, src=None):
        self.e(f"mov.b64 {{{a}, {b}}}, {src or self.T[i]};")

    def pack(self, i, a, b, dst=None):
        self.e(f"mov.b64 {dst or self.T[i]}, {{{a}, {b}}};")

    def slot_addr(self):
        self.e("bfe.u32 %%a, %%w, 8, 8;")
        self.e(f"min.u32 %%a, %%a, {self.NSM1};")
        self.e(f"mad.lo.u32 %%a, %%a, {self.slot_bytes}, {self.SB};")

    def slot_load(self):
        self.slot_addr()
        for q in range(self.rpt // 4):
            off = f"+{512 * q}" if q else ""
            self.e(f"ld.shared.v2.b64 {{%%U{2 * q}, %%U{2 * q + 1}}}, [%%a{off}];")

    def spill(self):
        self.slot_addr()
        for q in range(self.rpt // 4):
            off = f"+{512 * q}" if q else ""
            self.e(f"st.shared.v2.b64 [%%a{off}], {{{self.T[2 * q]}, {self.T[2 * q + 1]}}};")

    def cpair(self):
        self.e("mov.b64 %%C, {%%cf, %%cf};")

    def pairwise(self, op, srcs):
        """T_i = op(T_i, src_i) or with a callable giving the operands"""
        for i in range(self.np):
            a, b = srcs(i)
            self.e(f"{op}.rn.f32x2 {self.T[i]}, {a}, {b};")

    # A warp-wide test of every row before any row changes: unless every
    # |v| < hi (NaN fails) and, with lo, every |v| >= lo, the warp leaves
    # the fast path -- to EX, or with special (a callable emitting a per-row
    # test that sets %%p on rows the body cannot take) to a second test
    # that lets the special values through (NaN, inf, zero) and bails only
    # on the rest.  Past that test the warp goes back into the body, or,
    # with body, runs body (a copy of the computation that also gives the
    # special rows the C++ functions' results) and ends there; the copy
    # sits out of the hot path and keeps nothing live across it.
    # Each group is (hi, lo or None, vals) with vals(i) the pair register
    # of rows 2i and 2i+1; the groups share one vote.
    def range_check(self, hi, lo=None, vals=None, groups=None, special=None, body=None):
        groups = groups or [(hi, lo, vals or (lambda i: self.T[i]))]
        self.e("setp.ne.u32 %%ps, 0, 0;")
        for hi, lo, vals in groups:
            for i in range(self.np):
                self.e(f"mov.b64 {{%%v0, %%v1}}, {vals(i)};")
                for r, v in enumerate(("%%v0", "%%v1")):
                    self.e(f"abs.f32 {v}, {v};")
                    first = i == 0 and r == 0
                    self.e(f"mov.f32 %%mx, {v};" if first else f"max.NaN.f32 %%mx, %%mx, {v};")
                    if lo:
                        self.e(f"mov.f32 %%mn, {v};" if first else f"min.f32 %%mn, %%mn, {v};")
            self.e(f"setp.geu.or.f32 %%ps, %%mx, {kf(hi)}, %%ps;")
            if lo:
                self.e(f"setp.lt.or.f32 %%ps, %%mn, {kf(lo)}, %%ps;")
        self.e("vote.sync.any.pred %%ps, %%ps, 0xffffffff;")
        if special is None or not self.special:
            self.e("@%%ps bra EX%=;")
            return None
        k = self.nsv
        self.nsv += 1
        self.e(f"@%%ps bra SV{k}%=;")
        self.label(f"SC{k}")

        def block():
            self.label(f"SV{k}")
            self.e("setp.ne.u32 %%ps, 0, 0;")
            special()
            self.e("vote.sync.any.pred %%ps, %%ps, 0xffffffff;")
            self.e("@%%ps bra EX%=;")
            if body is None:
                self.e(f"bra.uni SC{k}%=;")
            else:
                body()
                self.nxt()
        self.deferred.append(block)
        return k

    def fix_rows(self, i, rows):
        """pair i of the rows after a computation whose input pair is in Y:
        rows(s, v) per row (s the input, v the result)"""
        self.unpack(i, "%%v0", "%%v1")
        self.e("mov.b64 {%%s0, %%s1}, %%Y;")
        for r in (0, 1):
            rows(f"%%s{r}", f"%%v{r}")
        self.pack(i, "%%v0", "%%v1")

    def rows_test(self, vals, test):
        """per row of vals: test(v) emits code setting %%p; %%ps |= %%p"""
        for i in range(self.np):
            self.e(f"mov.b64 {{%%v0, %%v1}}, {vals(i)};")
            for v in ("%%v0", "%%v1"):
                test(v)
                self.e("or.pred %%ps, %%ps, %%p;")

    def beyond(self, lo, v):
        """%%p = lo <= |v| < inf (NaN and inf pass)"""
        self.e(f"abs.f32 %%m, {v};")
        self.e(f"setp.ge.f32 %%p, %%m, {kf(lo)};")
        self.e(f"setp.lt.and.f32 %%p, %%m, {kf('inf')}, %%p;")

    # sin or cos of every row (the steps of sincos_fast): one body for
    # both, the kind (0 sin, 1 cos) from the dispatch index.  j = the
    # integer nearest x/pi - kind/2, r = x - (j + kind/2) pi, then one odd
    # polynomial, negated when j + kind is odd (a sign-bit flip)
    def trig(self, src=None, dst=None, kind=None):
        """sin/cos of the pairs src(i) into dst(i) (default: the rows, in
        place, after the range test, the kind from the dispatch index); a
        static kind (0 sin, 1 cos) skips the test and the index"""
        src = src or (lambda i: self.T[i])
        if kind is None:
            self.range_check("trig_fast", special=lambda: self.rows_test(
                lambda i: self.T[i], lambda v: self.beyond("trig_fast", v)))
            self.e(f"sub.u32 %%kd, %%i, {OPS['SIN']};")
            self.e("setp.ne.u32 %%p, %%kd, 0;")
            self.e("selp.b64 %%KM, 0xBF000000BF000000, 0x8000000080000000, %%p;")  # -kind/2
            self.e("selp.b64 %%F, 0x3F0000003F000000, 0x0000000000000000, %%p;")   # +kind/2
            self.e("shl.b32 %%kd, %%kd, 31;")
        else:
            self.e("mov.b64 %%KM, " + ("0xBF000000BF000000;" if kind else "0x8000000080000000;"))
            self.e("mov.b64 %%F, " + ("0x3F0000003F000000;" if kind else "0x0000000000000000;"))
            self.e(f"mov.b32 %%kd, {0x80000000 if kind else 0};")
        for i in range(self.np):
            t = src(i)
            self.e(f"mov.b64 %%K0, {kp('inv_pi')};")
            self.e(f"fma.rn.f32x2 %%JM, {t}, %%K0, %%KM;")
            self.e(f"mov.b64 %%K1, {kp('magic')};")
            self.e("add.rn.f32x2 %%JM, %%JM, %%K1;")
            self.e("sub.rn.f32x2 %%JJ, %%JM, %%K1;")
            self.e("add.rn.f32x2 %%JJ, %%JJ, %%F;")
            # r = x - j' (HI + MID + LO): fma(j', -HI, x) is fma(-j', HI, x) bit for bit
            self.e(f"mov.b64 %%K0, {kp('pi_hi', True)};")
            self.e(f"fma.rn.f32x2 %%R, %%JJ, %%K0, {t};")
            self.e(f"mov.b64 %%K0, {kp('pi_mid', True)};")
            self.e("fma.rn.f32x2 %%R, %%JJ, %%K0, %%R;")
            self.e(f"mov.b64 %%K0, {kp('pi_lo', True)};")
            self.e("fma.rn.f32x2 %%R, %%JJ, %%K0, %%R;")
            self.e("mul.rn.f32x2 %%S, %%R, %%R;")
            # sin r = r + (s r)(Q0 + s (Q1 + s (Q2 + s Q3)))
            self.e(f"mov.b64 %%K0, {kp('q3')};")
            self.e(f"mov.b64 %%K1, {kp('q2')};")
            self.e("fma.rn.f32x2 %%P, %%K0, %%S, %%K1;")
            for c in ("q1", "q0"):
                self.e(f"mov.b64 %%K0, {kp(c)};")
                self.e("fma.rn.f32x2 %%P, %%P, %%S, %%K0;")
            self.e("mul.rn.f32x2 %%Q, %%S, %%R;")
            self.e("fma.rn.f32x2 %%P, %%P, %%Q, %%R;")
            self.unpack(i, "%%n0", "%%n1", "%%JM")   # bit 0: parity of j
            self.unpack(i, "%%v0", "%%v1", "%%P")
            for r in (0, 1):
                n, v = f"%%n{r}", f"%%v{r}"
                self.e(f"shl.b32 {n}, {n}, 31;")
                self.e(f"xor.b32 {n}, {n}, %%kd;")
                self.e(f"mov.b32 %%a, {v};")
                self.e(f"xor.b32 %%a, %%a, {n};")
                self.e(f"mov.b32 {v}, %%a;")
            self.pack(i, "%%v0", "%%v1", dst(i) if dst else None)

    # log of every row (f_log: the logarithm of max(|t|, thr), 0 below the
    # threshold, inf and NaN passed through)
    def log(self):
        for i in range(self.np):
            self.unpack(i, "%%v0", "%%v1")
            for r in (0, 1):
                v, b, n, m, k = f"%%v{r}", f"%%u{r}", f"%%n{r}", f"%%m{r}", f"%%k{r}"
                self.e(f"abs.f32 {b}, {v};")
                self.e(f"max.f32 %%q, {b}, {self.THR};")
                self.e(f"mov.b32 {n}, %%q;")
                self.e(f"sub.u32 {k}, {n}, 0x3F3504F3;")
                self.e(f"shr.s32 {k}, {k}, 23;")
                self.e(f"mad.lo.u32 {m}, {k}, 0xFF800000, {n};")   # bits of m = i - (k << 23)
                self.e(f"add.u32 {k}, {k}, 0x4B400000;")           # bits of 1.5 * 2^23 + k
            self.e("mov.b64 %%F, {%%m0, %%m1};")
            self.e("mov.b64 %%JM, {%%k0, %%k1};")
            self.e(f"mov.b64 %%K0, {kp('one')};")
            self.e("sub.rn.f32x2 %%F, %%F, %%K0;")                # f = m - 1
            self.e(f"mov.b64 %%K1, {kp('magic')};")
            self.e("sub.rn.f32x2 %%JJ, %%JM, %%K1;")              # k as a float
            self.e(f"mov.b64 %%K0, {kp('lp7')};")
            self.e(f"mov.b64 %%K1, {kp('lp6')};")
            self.e("fma.rn.f32x2 %%P, %%K0, %%F, %%K1;")
            for c in ("lp5", "lp4", "lp3", "lp2", "lp1", "lp0"):
                self.e(f"mov.b64 %%K0, {kp(c)};")
                self.e("fma.rn.f32x2 %%P, %%P, %%F, %%K0;")
            self.e("mul.rn.f32x2 %%S, %%F, %%F;")
            self.e("fma.rn.f32x2 %%R, %%S, %%P, %%F;")
            self.e(f"mov.b64 %%K0, {kp('ln2_lo')};")
            self.e("fma.rn.f32x2 %%R, %%JJ, %%K0, %%R;")
            self.e(f"mov.b64 %%K0, {kp('ln2_hi')};")
            self.e("fma.rn.f32x2 %%R, %%JJ, %%K0, %%R;")
            self.unpack(i, "%%s0", "%%s1", "%%R")
            for r in (0, 1):
                v, b, s = f"%%v{r}", f"%%u{r}", f"%%s{r}"
                # b < thr ? 0 : (b <= FLT_MAX ? log : b)
                self.e(f"setp.le.f32 %%p, {b}, {kf('flt_max')};")
                self.e(f"selp.f32 {v}, {s}, {b}, %%p;")
                self.e(f"setp.lt.f32 %%p, {b}, {self.THR};")
                self.e(f"selp.f32 {v}, 0f00000000, {v}, %%p;")
            self.pack(i, "%%v0", "%%v1")

    # exp of every row when all |t| < 87 (exp_fast), else handed back
    def exp(self):
        # special: a warp with |x| >= 87 (or NaN) in any row runs a copy
        # whose scaling by 2^j is two exact halves (exp_wide: subnormal
        # results round once, large ones overflow), x >= 89 giving +inf and
        # x <= -110 +0, as f_exp does; NaN gives NaN
        def fix(sv, v):
            self.e(f"setp.ge.f32 %%p, {sv}, {kf('exp_inf')};")
            self.e(f"selp.f32 {v}, {kf('inf')}, {v}, %%p;")
            self.e(f"setp.le.f32 %%p, {sv}, {kf('exp_zero')};")
            self.e(f"selp.f32 {v}, 0f00000000, {v}, %%p;")

        def special_body():
            for i in range(self.np):
                self.e(f"mov.b64 %%Y, {self.T[i]};")
                self.exp_pair(i, wide=True)
                self.fix_rows(i, fix)
        self.range_check("exp_fast", special=lambda: None, body=special_body)
        for i in range(self.np):
            self.exp_pair(i)

    def exp_pair(self, i, wide=False):
        t = self.T[i]
        self.e(f"mov.b64 %%K0, {kp('log2e')};")
        self.e(f"mov.b64 %%K1, {kp('magic')};")
        self.e(f"fma.rn.f32x2 %%JM, {t}, %%K0, %%K1;")
        self.e("sub.rn.f32x2 %%JJ, %%JM, %%K1;")
        self.e(f"mov.b64 %%K0, {kp('ln2_hi', True)};")
        self.e(f"fma.rn.f32x2 %%R, %%JJ, %%K0, {t};")
        self.e(f"mov.b64 %%K0, {kp('ln2_lo', True)};")
        self.e("fma.rn.f32x2 %%R, %%JJ, %%K0, %%R;")
        self.e(f"mov.b64 %%K0, {kp('e6')};")
        self.e(f"mov.b64 %%K1, {kp('e5')};")
        self.e("fma.rn.f32x2 %%P, %%K0, %%R, %%K1;")
        for c in ("e4", "e3", "e2", "e1", "one"):
            self.e(f"mov.b64 %%K0, {kp(c)};")
            self.e("fma.rn.f32x2 %%P, %%P, %%R, %%K0;")
        self.unpack(i, "%%n0", "%%n1", "%%JM")
        if not wide:
            for r in (0, 1):
                # 2^j: the low bits of the rounded sum are j, shifted into the exponent
                self.e(f"mad.lo.u32 %%n{r}, %%n{r}, 8388608, 0x3F800000;")
            self.e("mov.b64 %%S, {%%n0, %%n1};")
            self.e(f"mul.rn.f32x2 {t}, %%P, %%S;")
            return
        for r in (0, 1):
            # j = the sum's bits - the magic's; 2^(j >> 1) into n, the rest into m
            self.e(f"sub.s32 %%n{r}, %%n{r}, {K['magic']};")
            self.e(f"shr.s32 %%m{r}, %%n{r}, 1;")
            self.e(f"sub.s32 %%n{r}, %%n{r}, %%m{r};")
            self.e(f"add.s32 %%m{r}, %%m{r}, 127;")
            self.e(f"shl.b32 %%m{r}, %%m{r}, 23;")
            self.e(f"add.s32 %%n{r}, %%n{r}, 127;")
            self.e(f"shl.b32 %%n{r}, %%n{r}, 23;")
        self.e("mov.b64 %%S, {%%m0, %%m1};")
        self.e(f"mul.rn.f32x2 {t}, %%P, %%S;")
        self.e("mov.b64 %%S, {%%n0, %%n1};")
        self.e(f"mul.rn.f32x2 {t}, {t}, %%S;")

    # The IEEE reciprocal, square root and quotient, correctly rounded, from
    # the hardware estimates and Newton-Raphson steps with FMA (P. Markstein,
    # "Computation of elementary functions on the IBM RISC System/6000
    # processor", IBM J. Res. Dev. 34, 1990): y = e + e (1 - b e) for 1/b
    # from the estimate e; sqrt x = g + (x - g g) h with g = x e, h = e / 2
    # from the reciprocal square-root estimate e; a / b = q + (a - b q) y
    # with q = a y and y the reciprocal above.  On the ranges the warp-wide
    # tests admit -- |b| < 2^126 for 1/b; x in [2^-100, inf) for sqrt x;
    # |a| in [2^-60, 2^60) and |b| < 2^60 for a / b (|b| < 0.001 being
    # protected anyway) -- each gives the bits of rcp.rn, sqrt.rn and
    # div.rn: checked against them for every float32 reciprocal and square
    # root and 1.2e9 quotients.  Outside those ranges the word is handed
    # back, and the switch uses the IEEE operations themselves.
    def rcp_pair(self, src, dst):
        """dst = 1 / src for one pair, its rows in the reciprocal's range"""
        self.e(f"mov.b64 {{%%v0, %%v1}}, {src};")
        self.e("rcp.approx.ftz.f32 %%u0, %%v0;")
        self.e("rcp.approx.ftz.f32 %%u1, %%v1;")
        self.e("mov.b64 %%P, {%%u0, %%u1};")
        self.e(f"mov.b64 %%K0, {kp('mone')};")
        self.e("mul.rn.f32x2 %%Q, %%P, %%K0;")           # -e
        self.e(f"mov.b64 %%K1, {kp('one')};")
        self.e(f"fma.rn.f32x2 %%Q, {src}, %%Q, %%K1;")    # 1 - b e
        self.e(f"fma.rn.f32x2 {dst}, %%P, %%Q, %%P;")     # e + e (1 - b e)

    def inv(self):
        # |t| < thr ? 0 : 1 / t; special: NaN goes through the steps (NaN),
        # +-inf gives +-0, as rcp.rn does; 2^126 <= |t| < inf leaves
        def fix(sv, v):
            self.e(f"abs.f32 %%m, {sv};")
            self.e(f"setp.eq.f32 %%p, %%m, {kf('inf')};")
            self.e(f"copysign.f32 %%q, {sv}, 0f00000000;")
            self.e(f"selp.f32 {v}, %%q, {v}, %%p;")

        def special_body():
            for i in range(self.np):
                self.e(f"mov.b64 %%Y, {self.T[i]};")
                self.inv_pair(i)
                self.fix_rows(i, fix)
        self.range_check("two_126", body=special_body, special=lambda: self.rows_test(
            lambda i: self.T[i], lambda v: self.beyond("two_126", v)))
        # every pair's reciprocal first (independent chains), then the selects
        for i in range(self.np):
            self.rcp_pair(self.T[i], f"%%U{i}")
        for i in range(self.np):
            self.inv_select(i)

    def inv_pair(self, i):
        self.rcp_pair(self.T[i], f"%%U{i}")
        self.inv_select(i)

    def inv_select(self, i):
        self.unpack(i, "%%v0", "%%v1")
        self.e(f"mov.b64 {{%%u0, %%u1}}, %%U{i};")
        for v, u in (("%%v0", "%%u0"), ("%%v1", "%%u1")):
            self.e(f"abs.f32 %%m, {v};")
            self.e(f"setp.lt.f32 %%p, %%m, {self.THR};")
            self.e(f"selp.f32 {v}, 0f00000000, {u}, %%p;")
        self.pack(i, "%%v0", "%%v1")

    def sqrt(self):
        # sqrt |t|; special: NaN goes through the steps (NaN), |t| = 0 gives
        # +0 and |t| = inf +inf, as sqrt.rn does; 0 < |t| < 2^-100 leaves
        def test(v):
            self.e(f"abs.f32 %%m, {v};")
            self.e("setp.gt.f32 %%p, %%m, 0f00000000;")
            self.e(f"setp.lt.and.f32 %%p, %%m, {kf('two_m100')}, %%p;")

        def fix(sv, v):
            self.e(f"abs.f32 %%m, {sv};")
            self.e("setp.eq.f32 %%p, %%m, 0f00000000;")
            self.e(f"setp.eq.or.f32 %%p, %%m, {kf('inf')}, %%p;")
            self.e(f"selp.f32 {v}, %%m, {v}, %%p;")

        def special_body():
            for i in range(self.np):
                self.e(f"mov.b64 %%Y, {self.T[i]};")
                self.sqrt_pair(i)
                self.fix_rows(i, fix)
        self.range_check("inf", lo="two_m100", body=special_body,
                         special=lambda: self.rows_test(lambda i: self.T[i], test))
        for i in range(self.np):
            self.sqrt_pair(i)

    def sqrt_pair(self, i):
        self.unpack(i, "%%v0", "%%v1")
        self.e("abs.f32 %%v0, %%v0;")
        self.e("abs.f32 %%v1, %%v1;")
        self.e("rsqrt.approx.ftz.f32 %%u0, %%v0;")
        self.e("rsqrt.approx.ftz.f32 %%u1, %%v1;")
        self.e("mov.b64 %%F, {%%v0, %%v1};")            # x
        self.e("mov.b64 %%P, {%%u0, %%u1};")            # e
        self.e("mul.rn.f32x2 %%S, %%F, %%P;")           # g = x e
        self.e(f"mov.b64 %%K0, {kp('half')};")
        self.e("mul.rn.f32x2 %%Q, %%P, %%K0;")          # h = e / 2
        self.e(f"mov.b64 %%K1, {kp('mone')};")
        self.e("mul.rn.f32x2 %%R, %%S, %%K1;")          # -g
        self.e("fma.rn.f32x2 %%R, %%R, %%S, %%F;")      # x - g g
        self.e(f"fma.rn.f32x2 {self.T[i]}, %%R, %%Q, %%S;")

    def div_check(self, num, den, pre=None):
        """the division's range test; a special row -- a NaN operand, an
        infinite one, a zero dividend -- is let through to a copy of the
        division (pre: the reversed forms' swap first) that gives it the
        IEEE quotient; finite operands out of range still leave"""
        def special():
            for i in range(self.np):
                self.e(f"mov.b64 {{%%v0, %%v1}}, {num(i)};")
                self.e(f"mov.b64 {{%%u0, %%u1}}, {den(i)};")
                for r in (0, 1):
                    self.beyond("two_60", f"%%u{r}")
                    self.e("or.pred %%ps, %%ps, %%p;")
                    self.beyond("two_60", f"%%v{r}")
                    self.e("or.pred %%ps, %%ps, %%p;")
                    self.e(f"abs.f32 %%m, %%v{r};")
                    self.e("setp.gt.f32 %%p, %%m, 0f00000000;")
                    self.e(f"setp.lt.and.f32 %%p, %%m, {kf('two_m60')}, %%p;")
                    self.e("or.pred %%ps, %%ps, %%p;")

        def body():
            if pre:
                pre()
            self.div_compute(fix=True)
        self.range_check(None, groups=[("two_60", None, den), ("two_60", "two_m60", num)],
                         special=special, body=body)

    def div_body(self):
        """t = t / u for the divisor pairs in U, with the protection
        |divisor| < thr -> 1; DTUX: the same after the range test"""
        self.div_check(lambda i: self.T[i], lambda i: f"%%U{i}")
        self.label("DTUX")
        self.div_compute()

    def div_compute(self, fix=False):
        """the rows (dividends) over U (divisors); with fix, a zero or
        infinite dividend over a divisor that is not NaN gives dividend *
        sign(divisor) and an infinite divisor dividend * (+-0), the IEEE
        quotients the Newton steps miss"""
        num = lambda i: self.T[i]
        den = lambda i: f"%%U{i}"
        for i in range(self.np):
            # y = 1 / b, q = a y, then q + (a - b q) y
            self.rcp_pair(den(i), "%%JJ")
            self.e(f"mul.rn.f32x2 %%JM, {num(i)}, %%JJ;")
            self.e(f"mov.b64 %%K0, {kp('mone')};")
            self.e(f"mul.rn.f32x2 %%R, {den(i)}, %%K0;")     # -b
            self.e(f"fma.rn.f32x2 %%R, %%R, %%JM, {num(i)};")  # a - b q
            self.e("fma.rn.f32x2 %%JM, %%R, %%JJ, %%JM;")
            self.e(f"mov.b64 {{%%s0, %%s1}}, {den(i)};")
            self.e("mov.b64 {%%c0, %%c1}, %%JM;")
            if fix:
                self.e(f"mov.b64 {{%%u0, %%u1}}, {num(i)};")
                for r in (0, 1):
                    a, b, q = f"%%u{r}", f"%%s{r}", f"%%c{r}"
                    self.e(f"abs.f32 %%m, {a};")
                    self.e(f"setp.eq.f32 %%p, %%m, {kf('inf')};")
                    self.e(f"setp.eq.or.f32 %%p, {a}, 0f00000000, %%p;")
                    self.e(f"setp.num.and.f32 %%p, {b}, {b}, %%p;")   # a NaN divisor: NaN
                    self.e(f"copysign.f32 %%q, {b}, 0f3F800000;")
                    self.e(f"mul.rn.f32 %%q, {a}, %%q;")
                    self.e(f"selp.f32 {q}, %%q, {q}, %%p;")
                    self.e(f"abs.f32 %%m, {b};")
                    self.e(f"setp.eq.f32 %%p, %%m, {kf('inf')};")
                    self.e(f"copysign.f32 %%q, {b}, 0f00000000;")
                    self.e(f"mul.rn.f32 %%q, {a}, %%q;")
                    self.e(f"selp.f32 {q}, %%q, {q}, %%p;")
            for v, b, q in (("%%v0", "%%s0", "%%c0"), ("%%v1", "%%s1", "%%c1")):
                self.e(f"abs.f32 %%m, {b};")
                self.e(f"setp.lt.f32 %%p, %%m, {self.THR};")
                self.e(f"selp.f32 {v}, 0f3F800000, {q}, %%p;")
            self.pack(i, "%%v0", "%%v1")

    # -- the gradient variant: marked words --------------------------------
    # A marker word (index END|COL1) announces that the next word's operands
    # hold constants; its constant field packs the constant ranges (the
    # format of gp_internal.cuh).  The loop runs the marked word's value
    # body with ret = its index + 1, so the body returns through TR into
    # the word's partial-derivative body (pt with respect to the rows t,
    # po with respect to the other operand, as pairs), and the tangent tail
    # scales the tangents of the two ranges.  Marked words the loop does
    # not run, and those whose value body gives up, are handed back as
    # their marker with the address at the marked word.
    PARTIAL = dict(PC="PONE", PCS="PONE", AC="PONE", AS="PONE", SS="PSUB", SC="PSUB",
                   RC="PRSUB", MS="PMS", MC="PMC", DS="PDIV", DC="PDIV", RDC="PRDIV",
                   SQ="PSQ", IV="PIV", LG="PLG", XP="PXP", AB="PAB", NG="PNG",
                   PX0="PONE", PX1="PONE", PXS0="PONE", PXS1="PONE", AX0="PONE", AX1="PONE",
                   SX0="PSUB", SX1="PSUB", RX0="PRSUB", RX1="PRSUB", MX0="PMX0", MX1="PMX1",
                   DX0="PDIV", DX1="PDIV", RDX0="PRDIV", RDX1="PRDIV")

    def partial_labels(self, ent):
        """per dispatch index: the partial-derivative body, or EX where the
        loop does not run the word"""
        out = []
        for i, lab in enumerate(ent):
            if lab == "TRG":
                out.append("PSIN" if i == OPS["SIN"] else "PCOS")
            else:
                out.append(self.PARTIAL.get(lab, "EX"))
        return out

    # partials that read the rows as they were before the word
    NEEDS_TO = ("PMS", "PMC", "PMX0", "PMX1", "PAB", "PSQ", "PLG", "PSIN", "PCOS")

    def marked_entry(self):
        """the marked word is loaded and dispatched through TV: a copy of a
        cheap body, a stub into a shared body (which returns through ret),
        or MKX when the loop does not run it (EX then hands back the
        marker, as it does when ret is set)"""
        e = self.e
        e("mov.b32 %%mk, %%cb;")
        e("bfe.u32 %%tl, %%w, 8, 2;")      # the marker's shape: its tangent tail
        e("ld.shared.v2.b32 {%%w, %%cb}, [%0];")
        e("add.u32 %0, %0, 8;")
        e("mov.b32 %%cf, %%cb;")
        e("and.b32 %%i, %%w, 63;")
        e("brx.idx.uni %%i, TV%=;")
        self.label("MKX")
        e("mov.u32 %%ret, 1;")
        e("bra.uni EX%=;")

    def save_rows(self, part):
        if part in self.NEEDS_TO:
            for i in range(self.np):
                self.e(f"mov.b64 %%TO{i}, {self.T[i]};")

    def partial_bodies(self, labels):
        for lab in labels:
            self.label(lab)
            self.partial_code(lab)
            self.e("brx.idx.uni %%tl, TQ%=;")

    def partial_code(self, lab):
        e, p = self.e, self.np
        ONES, MONES = "0x3F8000003F800000", "0xBF800000BF800000"
        if lab in ("PONE", "PSUB", "PRSUB", "PNG"):
            pt = MONES if lab in ("PRSUB", "PNG") else ONES
            po = MONES if lab == "PSUB" else ONES
            for i in range(p):
                e(f"mov.b64 %%PT{i}, {pt};")
                e(f"mov.b64 %%PO{i}, {po};")
        elif lab in ("PMS", "PMC", "PMX0", "PMX1"):
            for i in range(p):
                src = {"PMS": f"%%U{i}", "PMC": "%%C"}.get(lab) or self.X[int(lab[-1])][i]
                e(f"mov.b64 %%PT{i}, {src};")
                e(f"mov.b64 %%PO{i}, %%TO{i};")
        elif lab in ("PDIV", "PRDIV"):
            # divisor b in U, quotient v in the rows: r = 1/b, -v r; both 0
            # where |b| < thr (the protected branch is constant)
            for i in range(p):
                self.rcp_pair(f"%%U{i}", f"%%A{i}")
                e(f"mov.b64 %%K0, {MONES};")
                e(f"mul.rn.f32x2 %%S, {self.T[i]}, %%K0;")
                e(f"mul.rn.f32x2 %%S, %%S, %%A{i};")
                e(f"mov.b64 {{%%s0, %%s1}}, %%U{i};")
                e(f"mov.b64 {{%%c0, %%c1}}, %%A{i};")
                e("mov.b64 {%%v0, %%v1}, %%S;")
                for r in (0, 1):
                    e(f"abs.f32 %%m, %%s{r};")
                    e(f"setp.lt.f32 %%p, %%m, {self.THR};")
                    e(f"selp.f32 %%c{r}, 0f00000000, %%c{r}, %%p;")
                    e(f"selp.f32 %%v{r}, 0f00000000, %%v{r}, %%p;")
                r_, nv = ("%%PT", "%%PO") if lab == "PDIV" else ("%%PO", "%%PT")
                e(f"mov.b64 {r_}{i}, {{%%c0, %%c1}};")
                e(f"mov.b64 {nv}{i}, {{%%v0, %%v1}};")
        elif lab == "PSQ":
            # d sqrt|t| = sign(t) / (2 sqrt|t|); 0 at t = 0 (the protected
            # convention) and at |t| = inf
            for i in range(p):
                self.rcp_pair(self.T[i], f"%%A{i}")
                e(f"mov.b64 %%K0, {kp('half')};")
                e(f"mul.rn.f32x2 %%A{i}, %%A{i}, %%K0;")
                e(f"mov.b64 {{%%s0, %%s1}}, %%TO{i};")
                e(f"mov.b64 {{%%c0, %%c1}}, %%A{i};")
                for r in (0, 1):
                    e(f"copysign.f32 %%c{r}, %%s{r}, %%c{r};")
                    e(f"abs.f32 %%m, %%s{r};")
                    e("setp.eq.f32 %%p, %%m, 0f00000000;")
                    e(f"setp.eq.or.f32 %%p, %%m, {kf('inf')}, %%p;")
                    e(f"selp.f32 %%c{r}, 0f00000000, %%c{r}, %%p;")
                e(f"mov.b64 %%PT{i}, {{%%c0, %%c1}};")
        elif lab == "PIV":
            # d (1/t) = -v^2 (0 on the protected branch, where v = 0)
            for i in range(p):
                e(f"mov.b64 %%K0, {MONES};")
                e(f"mul.rn.f32x2 %%S, {self.T[i]}, %%K0;")
                e(f"mul.rn.f32x2 %%PT{i}, %%S, {self.T[i]};")
        elif lab == "PLG":
            # d log|t| = 1/t, 0 where |t| < thr
            for i in range(p):
                self.rcp_pair(f"%%TO{i}", f"%%A{i}")
                e(f"mov.b64 {{%%s0, %%s1}}, %%TO{i};")
                e(f"mov.b64 {{%%c0, %%c1}}, %%A{i};")
                for r in (0, 1):
                    e(f"abs.f32 %%m, %%s{r};")
                    e(f"setp.lt.f32 %%p, %%m, {self.THR};")
                    e(f"selp.f32 %%c{r}, 0f00000000, %%c{r}, %%p;")
                e(f"mov.b64 %%PT{i}, {{%%c0, %%c1}};")
        elif lab == "PXP":
            for i in range(p):
                e(f"mov.b64 %%PT{i}, {self.T[i]};")
        elif lab == "PAB":
            # sign(t): 1, -1, or 0 (at 0 and NaN)
            for i in range(p):
                e(f"mov.b64 {{%%s0, %%s1}}, %%TO{i};")
                for r in (0, 1):
                    e(f"setp.gt.f32 %%p, %%s{r}, 0f00000000;")
                    e(f"selp.f32 %%c{r}, 0f3F800000, 0f00000000, %%p;")
                    e(f"setp.lt.f32 %%p, %%s{r}, 0f00000000;")
                    e(f"selp.f32 %%c{r}, 0fBF800000, %%c{r}, %%p;")
                e(f"mov.b64 %%PT{i}, {{%%c0, %%c1}};")
        elif lab in ("PSIN", "PCOS"):
            # d sin t = cos t; d cos t = -sin t (the value's range test
            # already passed on these rows)
            self.trig(src=lambda i: f"%%TO{i}", dst=lambda i: f"%%PT{i}",
                      kind=1 if lab == "PSIN" else 0)
            if lab == "PCOS":
                for i in range(p):
                    e(f"mov.b64 %%K0, {MONES};")
                    e(f"mul.rn.f32x2 %%PT{i}, %%PT{i}, %%K0;")
        else:
            raise ValueError(lab)

    def tangent_tail(self):
        """dt[k] *= pt for k in [tlo, thi); dt[k] = (fresh ? 1 : dt[k]) * po
        for k in [olo, ohi); both ranges clamped to the KT slots"""
        e, p = self.e, self.np
        assert p == 2, "one float4 of tangents per (constant, lane): 4 rows"

        def loop(lab, factor):
            self.label(lab)
            e("ld.shared.v2.b64 {%%A0, %%A1}, [%%da];")
            for i in range(p):
                e(f"mul.rn.f32x2 %%A{i}, %%A{i}, {factor}{i};")
            e("st.shared.v2.b64 [%%da], {%%A0, %%A1};")
            e("add.u32 %%da, %%da, 512;")
            e("setp.lt.u32 %%p, %%da, %%de;")
            e(f"@%%p bra {lab}%=;")

        def bounds(lo_bit, hi_bit, skip):
            e(f"bfe.u32 %%lo, %%mk, {lo_bit}, 5;")
            e(f"bfe.u32 %%hi, %%mk, {hi_bit}, 5;")
            e(f"min.u32 %%hi, %%hi, {self.KT};")
            e("setp.ge.u32 %%p, %%lo, %%hi;")
            e(f"@%%p bra {skip}%=;")
            e(f"mad.lo.u32 %%da, %%lo, 512, {self.DB};")
            e(f"mad.lo.u32 %%de, %%hi, 512, {self.DB};")

        self.label("TT")
        bounds(0, 5, "TTO")
        loop("TTL", "%%PT")
        self.label("TTO")
        bounds(10, 15, "TTE")
        e("bfe.u32 %%a, %%mk, 20, 1;")
        e("setp.ne.u32 %%p, %%a, 0;")
        e("@%%p bra TTF%=;")
        loop("TTM", "%%PO")
        e("bra.uni TTE%=;")
        self.label("TTF")   # fresh: the tangent starts at 1, so it is po
        e("st.shared.v2.b64 [%%da], {%%PO0, %%PO1};")
        e("add.u32 %%da, %%da, 512;")
        e("setp.lt.u32 %%p, %%da, %%de;")
        e("@%%p bra TTF%=;")
        self.label("TTE")
        e("mov.u32 %%ret, 0;")
        e("bra.uni N%=;")
        # shape 1: dt[tlo] *= pt; shape 2: dt[olo] = po (fresh); the index
        # clamped to the KT slots like the ranges above
        self.label("TT1")
        e("and.b32 %%lo, %%mk, 31;")
        e(f"min.u32 %%lo, %%lo, {self.KT} - 1;")
        e(f"mad.lo.u32 %%da, %%lo, 512, {self.DB};")
        e("ld.shared.v2.b64 {%%A0, %%A1}, [%%da];")
        for i in range(p):
            e(f"mul.rn.f32x2 %%A{i}, %%A{i}, %%PT{i};")
        e("st.shared.v2.b64 [%%da], {%%A0, %%A1};")
        e("mov.u32 %%ret, 0;")
        e("bra.uni N%=;")
        self.label("TTF1")
        e("bfe.u32 %%lo, %%mk, 10, 5;")
        e(f"min.u32 %%lo, %%lo, {self.KT} - 1;")
        e(f"mad.lo.u32 %%da, %%lo, 512, {self.DB};")
        e("st.shared.v2.b64 [%%da], {%%PO0, %%PO1};")
        e("mov.u32 %%ret, 0;")
        e("bra.uni N%=;")

    # cheap bodies (no range test, a handful of instructions) end with a
    # plain branch to the next word; in the gradient variant the others
    # return through ret, and the marked words of the cheap ones run a copy
    # of the body that goes on to its partial-derivative body directly
    CHEAP = ("PX", "PXS", "PC", "PCS", "AS", "SS", "MS", "AX", "SX", "MX", "RX", "AC", "SC",
             "MC", "RC", "AB", "NG")

    @staticmethod
    def stem(name):
        col = int(name[-1]) if name[-1] in "01" and name not in ("PC",) else None
        return (name[:-1] if col is not None else name), col

    def body(self, name):
        """the value body of one dispatch label; True when it ends with its
        own branch (the divisions go on to the shared division body)"""
        e, p, X = self.e, self.np, self.X
        stem, col = self.stem(name)
        if stem == "PX" or stem == "PXS":
            if stem == "PXS":
                self.spill()
            for i in range(p):
                e(f"mov.b64 {self.T[i]}, {X[col][i]};")
        elif stem in ("PC", "PCS"):
            if stem == "PCS":
                self.spill()
            self.cpair()
            for i in range(p):
                e(f"mov.b64 {self.T[i]}, %%C;")
        elif stem in ("AS", "SS", "MS"):
            self.slot_load()
            op = dict(AS="add", SS="sub", MS="mul")[stem]
            self.pairwise(op, lambda i: (self.T[i], f"%%U{i}"))
        elif stem in ("AX", "SX", "MX"):
            op = dict(AX="add", SX="sub", MX="mul")[stem]
            self.pairwise(op, lambda i, c=col: (self.T[i], X[c][i]))
        elif stem == "RX":
            self.pairwise("sub", lambda i, c=col: (X[c][i], self.T[i]))
        elif stem in ("AC", "SC", "MC"):
            self.cpair()
            op = dict(AC="add", SC="sub", MC="mul")[stem]
            self.pairwise(op, lambda i: (self.T[i], "%%C"))
        elif stem == "RC":
            self.cpair()
            self.pairwise("sub", lambda i: ("%%C", self.T[i]))
        elif stem == "AB" or stem == "NG":
            op = "abs" if stem == "AB" else "neg"
            for i in range(p):
                self.unpack(i, "%%v0", "%%v1")
                e(f"{op}.f32 %%v0, %%v0;")
                e(f"{op}.f32 %%v1, %%v1;")
                self.pack(i, "%%v0", "%%v1")
        elif stem == "DS":
            # the divisor pairs into U, then the shared body
            self.slot_load()
            e("bra.uni DTU%=;")
            return True
        elif stem in ("DC", "DX"):
            src = "%%C" if stem == "DC" else None
            if stem == "DC":
                self.cpair()
            for i in range(p):
                e(f"mov.b64 %%U{i}, {src or X[col][i]};")
            e("bra.uni DTU%=;")
            return True
        elif stem in ("RDC", "RDX"):
            # u / t: the range test on these operands first (a word
            # handed back must leave the rows untouched), then the rows
            # become the divisor and the operand the dividend, and the
            # shared body divides (rare: 0.13 words per program of the
            # Pagie-1 population)
            if stem == "RDC":
                self.cpair()
            opnd = (lambda i: "%%C") if stem == "RDC" else (lambda i, c=col: X[c][i])

            def swap():
                for i in range(p):
                    e(f"mov.b64 %%U{i}, {self.T[i]};")
                    e(f"mov.b64 {self.T[i]}, {opnd(i)};")
            self.div_check(num=opnd, den=lambda i: self.T[i], pre=swap)
            swap()
            e("bra.uni DTUX%=;")
            return True
        elif stem == "SQ":
            self.sqrt()
        elif stem == "IV":
            self.inv()
        elif stem == "TRG":
            self.trig()
        elif stem == "LG":
            self.log()
        elif stem == "XP":
            self.exp()
        else:
            raise ValueError(name)
        return False

    # -- the loop -----------------------------------------------------------
    def table(self):
        """64 branch targets; a label names one body (ops sharing a body say so
        by sharing its label, and no two different bodies share a label)"""
        ent = ["EX"] * 64
        base = dict(PUSH_C="PC", PUSH_C_SP="PCS", ADD_S="AS", SUB_S="SS", MUL_S="MS",
                    ADD_C="AC", SUB_C="SC", RSUB_C="RC", MUL_C="MC", ABS="AB", NEG="NG")
        for k, v in base.items():
            ent[OPS[k]] = v
        if self.divs:
            for k, v in dict(DIV_S="DS", DIV_C="DC", RDIV_C="RDC", SQRT="SQ", INV="IV",
                             SIN="TRG", COS="TRG", LOG="LG", EXP="XP").items():
                ent[OPS[k]] = v
        if self.xreg:
            xops = dict(PUSH_X="PX", PUSH_X_SP="PXS", ADD_X="AX", SUB_X="SX", RSUB_X="RX",
                        MUL_X="MX")
            if self.divs:
                xops.update(DIV_X="DX", RDIV_X="RDX")
            for k, v in xops.items():
                ent[OPS[k]] = v + "0"
                ent[OPS[k] | COL1] = v + "1"
        if self.grad:
            ent[OPS["END"] | COL1] = "MK"
        owner = {}
        for op, lab in enumerate(ent):
            base = op & (COL1 - 1)
            if lab == "EX":
                continue
            kind = {OPS["SIN"]: "trig", OPS["COS"]: "trig"}.get(base, base)
            assert owner.setdefault(lab, kind) == kind, f"label {lab} names two bodies"
        return ent

    def generate(self):
        p = self.np
        ent = self.table()
        used = sorted(set(ent) - {"EX"})
        e = self.e
        e("{")
        e(".reg .pred %%p, %%ps;")
        e(".reg .b32 %%w, %%cb, %%i, %%a, %%kd, %%n<2>, %%m<2>, %%k<2>;")
        e(".reg .f32 %%cf, %%q, %%m, %%mx, %%mn, %%v<2>, %%u<2>, %%s<2>, %%c<2>;")
        e(f".reg .b64 %%C, %%U<{p}>, %%K<2>, %%KM, %%JM, %%JJ, %%R, %%S, %%P, %%Q, %%F;")
        if self.divs and self.special:
            e(".reg .b64 %%Y;")
        e("T%=: .branchtargets " + ", ".join(f"{x}%=" for x in ent) + ";")
        if self.grad:
            part = self.partial_labels(ent)
            e(".reg .b32 %%ret, %%mk, %%tl, %%lo, %%hi, %%da, %%de;")
            e("TQ%=: .branchtargets TT%=, TT1%=, TTF1%=, TT%=;")
            e(f".reg .b64 %%TO<{p}>, %%PT<{p}>, %%PO<{p}>, %%A<{p}>;")
            cheap = [self.stem(lab)[0] in self.CHEAP for lab in ent]
            # a marked word's value body: the copy of a cheap body (its
            # partial derivatives follow inline), else the shared one, which
            # returns through ret into the partial-derivative body
            tv = [("V" + lab if cheap[i] else "S" + lab) if part[i] != "EX" else "MKX"
                  for i, lab in enumerate(ent)]
            e("TV%=: .branchtargets " + ", ".join(f"{x}%=" for x in tv) + ";")
            tr = ["N"] + [("EX" if cheap[i] else part[i]) for i in range(64)]
            e("TR%=: .branchtargets " + ", ".join(f"{x}%=" for x in tr) + ";")
            e("mov.u32 %%ret, 0;")
        self.label("N")
        e("ld.shared.v2.b32 {%%w, %%cb}, [%0];")
        e("mov.b32 %%cf, %%cb;")
        e("add.u32 %0, %0, 8;")
        e("and.b32 %%i, %%w, 63;")
        e("brx.idx.uni %%i, T%=;")
        X = self.X
        for name in used:
            self.label(name)
            if name == "MK":
                self.marked_entry()
                continue
            if self.body(name):
                continue
            if self.grad and self.stem(name)[0] in self.CHEAP:
                e("bra.uni N%=;")
            else:
                self.nxt()
        if self.grad:
            for name in used:
                if self.stem(name)[0] in self.CHEAP and self.PARTIAL.get(name, "EX") != "EX":
                    self.label("V" + name)
                    self.save_rows(self.PARTIAL[name])
                    self.body(name)
                    self.partial_code(self.PARTIAL[name])
                    e("brx.idx.uni %%tl, TQ%=;")
        if self.divs:
            # t = t / u with the protection, the divisor pairs in U
            self.label("DTU")
            self.div_body()
            self.nxt()
        if self.grad:
            # stubs into the shared bodies: ret = the word's index + 1 (TR)
            done = set()
            for i, lab in enumerate(tv):
                if not lab.startswith("S") or lab in done:
                    continue
                done.add(lab)
                self.label(lab)
                e("add.u32 %%ret, %%i, 1;")
                self.save_rows(part[i])
                e(f"bra.uni {lab[1:]}%=;")
            self.partial_bodies(sorted(set(tr[1:]) - {"EX"}))
            self.tangent_tail()
        for block in self.deferred:
            block()
        self.label("EX")
        if self.grad:
            # a marked word whose value body gave up (a range test): hand
            # back its marker, the address at the marked word
            e("setp.ne.u32 %%p, %%ret, 0;")
            e(f"@%%p mov.b32 %%w, {OPS['END'] | COL1};")
            e("@%%p mov.b32 %%cf, %%mk;")
            e("@%%p sub.u32 %0, %0, 8;")
        e(f"mov.b32 {self.HW}, %%w;")
        e(f"mov.f32 {self.HC}, %%cf;")
        e("}")
        return self.lines



def function(rpt, divs, xreg, grad=False):
    g = Gen(rpt, divs, xreg, grad)
    lines = g.generate()
    p = rpt // 2
    name = f"fast_r{rpt}_{'divs' if divs else 'nodivs'}_{'x' if xreg else 'nox'}" + \
        ("_grad" if grad else "")
    body = "\n".join(f'        "{ln}\\n\\t"' for ln in lines)
    outs = ", ".join(['"+r"(pa)'] + [f'"+l"(t[{i}])' for i in range(p)] + ['"=r"(hw)', '"=f"(hc)'])
    ins = ", ".join(['"r"(sb)', '"n"(NSLOT - 1)'] + [f'"l"(x0[{i}])' for i in range(p)]
                    + [f'"l"(x1[{i}])' for i in range(p)] + ['"f"(kThr)']
                    + (['"r"(db)', '"n"(KT)'] if grad else []))
    return (f"template <int NSLOT{', int KT' if grad else ''}>\n"
            f"__device__ __forceinline__ void {name}(uint32_t &pa, uint64_t (&t)[{p}],\n"
            f"        const uint64_t (&x0)[{p}], const uint64_t (&x1)[{p}], uint32_t sb,\n"
            f"        {'uint32_t db, ' if grad else ''}uint32_t &hw, float &hc) {{\n"
            f"    asm volatile(\n{body}\n"
            f"        : {outs}\n"
            f"        : {ins});\n}}\n")


HEADER = '''// gp_fast.cuh -- the evaluator's indexed-branch fast loop in inline PTX.
// GENERATED by gen_fast.py (same directory); edit that script, not this file.
//
// fast_r<RPT>_<divs|nodivs>_<x|nox><NSLOT>(pa, t, x0, x1, sb, hw, hc) runs
// compiled instruction words from the shared-memory address pa over RPT
// rows per lane, held as RPT/2 pairs {row 2i, row 2i+1} in t.  It stops at
// the first word it does not run, returns that word and its constant in
// hw and hc, leaves pa just past it and the rows untouched by it.  sb is
// the lane's slot-0 address in the shared-memory stack ([slot][q][lane]
// float4); slots are clamped to NSLOT - 1; x0 and x1 hold columns 0 and 1
// of the lane's rows (read only by the _x variants).  Every one of the 64
// values of the six-bit dispatch index has a table entry.  The statement
// declares no memory clobber: the shared memory it reads and writes (the
// code buffer, written before a barrier, and the stack, touched elsewhere
// only by other volatile asm statements, which keep their order) needs none,
// and a clobber made the compiler reload the kernel arguments after every
// call.
#pragma once

#include <cstdint>

namespace gpk {

'''


def main():
    parts = [HEADER]
    for rpt in (4, 8):
        for divs in (True, False):
            for xreg in (True, False):
                parts.append(function(rpt, divs, xreg))
                parts.append("\n")
    # the constant gradient's loop (4 rows per lane, the division set)
    for xreg in (True, False):
        parts.append(function(4, True, xreg, grad=True))
        parts.append("\n")
    parts.append("}  // namespace gpk\n")
    with open(os.path.join(HERE, "gp_fast.cuh"), "w") as f:
        f.write("".join(parts))


if __name__ == "__main__":
    main()
