"""Per-element error bounds for the tensor-core GEMM stages.

The GEMM stages accumulate in f32 on the tensor cores: an output is the sum of
its K products taken one MMA instruction at a time (16 bf16 or 32 e4m3
products per instruction, in k order) into an accumulator that starts at zero
at the beginning of every K-chunk (chunk_cols below); the chunk partials are
then added in chunk order in f32.

Model of one instruction (products of bf16 or e4m3 operands are exact in f32):
the accumulator d and the t products are aligned to the largest of them and
the result is normalised to 24 significant bits, so each of the t + 1 terms and
the result can be off by at most one unit in the 24th bit of the largest
magnitude: |error| <= (t + 2) 2^-23 (|d| + sum |p|).  With t = 16 this is
36 u (|d| + sum |p|), u = 2^-24; the e4m3 instructions (t = 32) get 68 u.
Summed over the instructions of a chunk with |d| bounded by the exact partial
sum plus the error so far, this gives a bound that follows the data (partial
sums of random-signed products grow like the square root of their count)
instead of the worst case K u sum|w x| of a serial sum, which at K = 37632 is
larger than the outputs themselves.

Everything here is test tolerance arithmetic on exact (FP64) values computed
from the oracle's results; it shares nothing with the CUDA path.
"""
import numpy as np

U = 2.0 ** -24
# terms aligned per instruction + the result, each within 2^-23 = 2 u of the largest
C_MMA = {16: 36.0, 32: 68.0}


def chunk_cols(K: int, N: int) -> int:
    """The K-chunk the stage uses for a layer of N outputs: two chunks for 8 or
    more tiles of 128 output rows and K >= 512; otherwise the whole K up to 1024
    columns, above that as few equal chunks as give about 64 units of 128
    output rows, at most one per 1024 columns; chunks rounded up to 128
    columns."""
    mt = (N + 127) // 128
    if mt >= 8 and K >= 512:
        return ((K + 1) // 2 + 127) // 128 * 128
    if K <= 1024:
        return K
    c = max(1, min((K + 1023) // 1024, (64 + mt - 1) // mt))
    return ((K + c - 1) // c + 127) // 128 * 128


def mma_bound(x, xe, w, kstep: int):
    """Exact sums A = x @ w.T and a bound E on |acc_gpu - A| per element.

    x   [n, K] the oracle's input values (exact), xe [n, K] >= 0 a bound on
        |x_gpu - x| (zeros when the GPU's input equals the oracle's);
    w   [N, K] weights (exact values of the operand codes);
    kstep products per MMA instruction (16 for bf16, 32 for e4m3)."""
    x = np.asarray(x, np.float64)
    xe = np.asarray(xe, np.float64)
    w = np.asarray(w, np.float64)
    n, K = x.shape
    N = w.shape[0]
    kc = chunk_cols(K, N)
    c = C_MMA[kstep] * U
    aw = np.abs(w)
    A = np.zeros((n, N))
    E = np.zeros((n, N))
    for q in range(n):
        s_exact = np.zeros(N)
        s_err = np.zeros(N)
        for ci, k0 in enumerate(range(0, K, kc)):
            k1 = min(K, k0 + kc)
            m = (k1 - k0) // kstep
            p = (w[:, k0:k1] * x[q, k0:k1]).reshape(N, m, kstep).sum(-1)         # exact per instruction
            pa = (aw[:, k0:k1] * (np.abs(x[q, k0:k1]) + xe[q, k0:k1])).reshape(N, m, kstep).sum(-1)
            pe = (aw[:, k0:k1] * xe[q, k0:k1]).reshape(N, m, kstep).sum(-1)     # input perturbation
            D = np.cumsum(p, axis=1)
            De = np.cumsum(pe, axis=1)
            e = np.zeros(N)
            for k in range(m):
                dprev = (np.abs(D[:, k - 1]) + De[:, k - 1] + e) if k > 0 else 0.0
                e = e + c * (dprev + pa[:, k])
            ch_val = D[:, -1]
            ch_err = e + De[:, -1]
            # chunk partials are added in chunk order in f32, from zero
            s_exact = s_exact + ch_val
            s_err = s_err + ch_err + (U * (np.abs(s_exact) + s_err + ch_err) if ci > 0 else 0.0)
        A[q] = s_exact
        E[q] = s_err
    return A, E


GELU_LIP = 1.13   # max |gelu'| = 1.1289...


def gelu_f32_eval(v_abs, g_abs):
    """Bound on the f32 evaluation error of 0.5 v (1 + erf(v / sqrt 2)):
    erff within 2 ulp (CUDA's documented bound), three roundings."""
    return 4 * U * v_abs + 2 * U * g_abs + 1e-38


def rne_interval(orc_round, val, err):
    """The rounded GPU value lies in [round(val - err), round(val + err)]
    (rounding is monotone); returns the bound on |gpu_rounded - round(val)|."""
    r = orc_round(val)
    lo = orc_round(val - err)
    hi = orc_round(val + err)
    return r, np.maximum(np.abs(hi - r), np.abs(r - lo))


def determined_prefix(z, e, k):
    """Rank positions fixed by the intervals [z - e, z + e] of one row each.

    The set of the top r + 1 entries is fixed when the smallest lower end in
    it exceeds the largest upper end outside it; position r is fixed when the
    sets of the top r and top r + 1 are.  Returns (order [n, k] of the exact
    values, sets_fixed [n, k], pos_fixed [n, k]) with ties broken by index."""
    z = np.asarray(z, np.float64)
    e = np.asarray(e, np.float64)
    n, M = z.shape
    order = np.lexsort((np.tile(np.arange(M), (n, 1)), -z), axis=1)
    sets = np.zeros((n, k), bool)
    for q in range(n):
        o = order[q]
        lo_in = np.minimum.accumulate((z[q] - e[q])[o])
        hi_out = np.maximum.accumulate(((z[q] + e[q])[o])[::-1])[::-1]
        for r in range(k):
            sets[q, r] = lo_in[r] > hi_out[r + 1]
    pos = sets.copy()
    pos[:, 1:] &= sets[:, :-1]
    return order[:, :k], sets, pos


def check_topk(idx_gpu, z, e, k):
    """Asserts the GPU's top-k indices agree with the exact values wherever
    the intervals fix them; returns how many rows have all k positions fixed."""
    order, sets, pos = determined_prefix(z, e, k)
    idx_gpu = np.asarray(idx_gpu)[:, :k]
    for q in range(order.shape[0]):
        for r in range(k):
            if pos[q, r]:
                assert idx_gpu[q, r] == order[q, r], (q, r, idx_gpu[q], order[q])
            if sets[q, r]:
                assert set(idx_gpu[q, :r + 1]) == set(order[q, :r + 1]), (q, r)
    return int(np.sum(pos.all(axis=1)))


def bf16_layer_bracket(orc, x, w, act):
    """A tensor-core bf16 layer on input x (the GPU's own input values): the
    oracle's value act(w x) and the interval [lo, hi] in which the GPU's
    bf16-rounded output must lie (f32 accumulation within the instruction
    model, the f32 GELU within its evaluation bound, then monotone rounding)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    A, E = mma_bound(x, np.zeros_like(x), w, 16)
    if act == 2:
        G = orc.linear(x, w, 2)
        d = GELU_LIP * E + gelu_f32_eval(np.abs(A) + E, np.abs(G) + GELU_LIP * E)
    elif act == 1:
        G = orc.linear(x, w, 1)
        d = E
    else:
        G = orc.linear(x, w, 0)
        d = E
    return G, orc.round_bf16(G - d), orc.round_bf16(G + d)


def logits_bound(orc, x, w, kstep=16, vscale=1.0):
    """A final tensor-core layer (f32 logits, no activation) on input x: the
    oracle's logits and the per-element bound on the GPU's deviation."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    A, E = mma_bound(x, np.zeros_like(x), w, kstep)
    if vscale == 1.0:
        return orc.linear(x, w, 0), E
    z = A * vscale
    return z, vscale * E + U * np.abs(z) + U * vscale * E


def e4m3_layer_bracket(orc, xq, wq, vscale, act, s_out):
    """An FP8 layer on the GPU's own input codes xq (values): the oracle's
    output code value and the interval of codes the GPU may produce
    (v = act(f32(acc * vscale)), code = e4m3(f32(v / s_out)), monotone)."""
    A, E = mma_bound(xq, np.zeros_like(xq), wq, 32)
    _, own, _ = orc.linear_fp8(xq, wq, vscale, act, s_out)
    V = A * vscale
    dv = vscale * E + U * vscale * (np.abs(A) + E)
    f = (lambda t: np.maximum(t, 0.0)) if act == 1 else (lambda t: t)
    code = lambda t: orc.round_e4m3(orc.round_f32(orc.round_f32(f(t)) / s_out))
    return own, code(V - dv), code(V + dv)
