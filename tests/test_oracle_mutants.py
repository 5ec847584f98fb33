"""Planted mistakes: the oracle's pins catch a plausible error anywhere in it.

Each case copies the oracle's modules into a fresh package with ONE expression changed (a wrong
sign, a dropped term, an index off by one, a transposed operand) and runs the pins of
test_oracle_dd / test_oracle_ozaki / test_oracle_refine against the copy.  At least one pin
must fail one of its checks; a copy that only makes pins crash is not counted as caught.  The
stored regression of workload 0 is left out: it repeats the oracle's own
output, so it would catch every change and pin nothing.  Everything runs on the CPU; the
oracle itself is never modified.
"""
import os
import sys
import types

import pytest

from tests import test_oracle_dd as tdd
from tests import test_oracle_ozaki as toz
from tests import test_oracle_refine as trf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODULES = ("ddarith", "ozaki", "refine", "truth")

# (module, original text, planted text, what the mistake is)
MUTANTS = [
    ("ddarith", "y = (a - (x - z)) + (b - z)", "y = (a - (x - z)) - (b - z)", "TwoSum: wrong sign"),
    ("ddarith", "e = ((ah * bh - p) + ah * bl + al * bh) + al * bl", "e = ((ah * bh - p) + ah * bl + al * bh)",
     "TwoProduct: dropped lo*lo term"),
    ("ddarith", "    cl = bl + t\n", "    cl = bl\n", "pair arithmetic: dropped TwoSum error"),
    ("ddarith", "    se = se + al\n", "    se = se\n", "dd + d: dropped low word"),
    ("ozaki", "e + 1 - DIGIT_BITS * r))", "e - DIGIT_BITS * r))", "plane weight: exponent off by one"),
    ("ozaki", "d = np.rint(res / ws)", "d = np.floor(res / ws)", "digits: truncation instead of round to nearest"),
    ("ozaki", "S[t] = S[t] + P if t in S else P", "S[t] = P", "anti-diagonal sum: dropped pairs"),
    ("ozaki", "if r + s <= T]", "if r + s < T]", "pair set: last anti-diagonal dropped"),
    ("ozaki", "eL + eR + 2 - DIGIT_BITS * t", "eL + eR + 1 - DIGIT_BITS * t", "recombination: scale off by one"),
    ("ozaki", "return np.transpose(d, (0, 2, 1)), f, res.T", "return d, f, res.T",
     "column slicing: transposed digit planes"),
    ("ozaki", "f + beta)))", "f + beta + 1)))", "tau: exponent off by one"),
    ("ozaki", "hi, lo = dd.dd_add_d(hi, lo, term)", "hi, lo = dd.dd_add_d(hi, 0.0 * lo, term)",
     "recombination: low word dropped"),
    ("refine", "diff = lam[None, :] - lam[:, None]", "diff = lam[:, None] - lam[None, :]",
     "correction: wrong sign of the eigenvalue gap"),
    ("refine", "np.fill_diagonal(E, r / 2.0)", "np.fill_diagonal(E, r)", "correction: diagonal r instead of r/2"),
    ("refine", "r = dd.dd_add_d(-nh, -nl, 1.0)[0]", "r = dd.dd_add_d(nh, nl, -1.0)[0]", "r: wrong sign"),
    ("refine", "Wp = oz.ozaki_product(X1.T, Res,", "Wp = oz.ozaki_product(X1, Res,", "W: transposed operand"),
    ("refine", "ch, cl = dd.pair_add(X1, Up[\"hi\"], Up[\"lo\"])", "ch, cl = dd.pair_add(X, Up[\"hi\"], Up[\"lo\"])",
     "update: X instead of X^(1)"),
    ("refine", "math.sqrt((xi * delta * g) / (Lam * S2)) / (0.75 * U)", "math.sqrt((xi * delta * g) / (Lam * S2)) / U",
     "beta: dropped 0.75 of tau"),
    ("refine", "return 53 - beta + ceil_log2_sqrt(n)", "return 53 - beta + ceil_log2_int(n)",
     "alpha: log2 n for log2 sqrt n"),
    ("refine", "- SLICE_MARGIN_LOG2) >= float(n)", "- SLICE_MARGIN_LOG2 - 1) >= float(n)",
     "slice rule: margin off by one bit"),
    ("refine", "oz.DIGIT_BITS * k - int(eL) - int(eR)", "oz.DIGIT_BITS * k - int(eL)",
     "slice rule: right operand's exponent dropped"),
    ("refine", "E[i, j] = -sh / 2.0", "E[i, j] = sh / 2.0", "cluster rule: wrong sign of r_ij"),
    ("refine", "est = step_norm * step_norm * Lam_new", "est = step_norm * Lam_new", "stopping test: dropped square"),
    ("refine", "    s = np.sort(lam)\n", "    s = lam\n", "min gap: estimates not sorted"),
    ("refine", "g = float(np.min(gaps)) if gaps.size else Lam", "g = float(np.max(gaps)) if gaps.size else Lam",
     "min gap: largest gap instead of the smallest"),
    ("refine", "gaps = gaps[gaps > omega]", "gaps = gaps[gaps >= omega]", "min gap: gaps equal to omega kept"),
    ("refine", "Lam = float(np.max(np.abs(lam)))", "Lam = float(np.max(lam))", "max |lam|: absolute value dropped"),
    ("refine", "math.ldexp(1.0, 2 * int(x))", "math.ldexp(1.0, int(x))", "S2: 2^f instead of 2^(2f)"),
    ("truth", "    Y = Xhat * s[None, :]\n", "    Y = Xhat\n", "forward error: no sign alignment"),
    ("truth", "return float(np.linalg.norm(dh + dl, 2))", "return float(np.linalg.norm(dh + dl))",
     "forward error: Frobenius norm for the 2-norm"),
    ("truth", "dh, dl = dd.dd_add(Xh, Xl, -Y, np.zeros_like(Y))", "dh, dl = dd.dd_add(Xh, 0.0 * Xl, -Y, np.zeros_like(Y))",
     "forward error: low word of X dropped"),
    ("truth", "Qh, _ = np.linalg.qr(np.asarray(Xhat)[:, cols])", "Qh = np.asarray(Xhat)[:, cols]",
     "subspace error: columns of X^ not orthonormalised"),
    ("truth", "return float(np.linalg.norm(P, 2))", "return float(np.linalg.norm(P))",
     "subspace error: Frobenius norm for the 2-norm"),
    ("ddarith", "    q2 = rh / bh\n", "    q2 = 0.0 * rh / bh\n", "dd division: Newton correction dropped"),
    ("ddarith", "sh, sl = dd_add(sh, sl, h[k], l[k])", "sh, sl = dd_add(sh, sl, h[k], 0.0 * l[k])",
     "dd sum: low words dropped"),
    ("refine", "b = floor_log2(q) if opts.beta_rounding == \"floor\" else ceil_log2f(q)",
     "b = ceil_log2f(q) if opts.beta_rounding == \"floor\" else floor_log2(q)", "beta: ceiling for the floor"),
    ("refine", "return (2 ** 31 - 1) // (n * oz.DIGIT_MAX * oz.DIGIT_MAX)",
     "return (2 ** 32 - 1) // (n * oz.DIGIT_MAX * oz.DIGIT_MAX)", "int32 plane bound: 2^32 for 2^31"),
    ("refine", "xi=float(min(kmax * kmax, n))", "xi=float(min(kmax, n))", "sparse rule: k for k^2"),
    ("refine", "53 - beta + ceil_log2_int(kmax)", "53 - beta + ceil_log2_int(kmax + 1)",
     "sparse rule: alpha from k + 1"),
    ("refine", "beta = 54 - oz.DIGIT_BITS * opts.x_planes", "beta = 53 - oz.DIGIT_BITS * opts.x_planes",
     "previous-study form: beta off by one"),
    ("refine", "        X1 = X - resid\n", "        X1 = X\n", "previous-study form: X not cut to its planes"),
    ("refine", "sX = -(-(54 - beta) // oz.DIGIT_BITS)", "sX = (54 - beta) // oz.DIGIT_BITS",
     "s_X: floor for the ceiling"),
    ("ozaki", "for s in range(1, kR + 1) if r + s <= T]", "for s in range(1, kR) if r + s <= T]",
     "pair set: last plane of the right operand dropped"),
    ("ddarith", "    y = b - (x - a)\n", "    y = b + (x - a)\n", "fast TwoSum: wrong sign"),
    ("ddarith", "    pe = pe + al * b\n", "    pe = pe\n", "dd * d: low word dropped"),
    ("ddarith", "            e = e + Ll[:, k:k + 1] * b\n", "            e = e\n", "dd matmul: low words of L dropped"),
    ("ddarith", "    hi = c - (c - a)\n", "    hi = c - (c + a)\n", "Veltkamp split: wrong sign"),
    ("ozaki", "e = np.where(fr == 0.5, ex - 1, ex).astype(np.int64)", "e = ex.astype(np.int64)",
     "exponent: powers of two one too high"),
    ("ozaki", "return ceil_log2(np.max(np.abs(M), axis=1))", "return ceil_log2(np.max(M, axis=1))",
     "exponent: absolute value dropped"),
    ("ozaki", "0.75 * np.ldexp(1.0, np.where(e == EZERO, 0, e + 54 - DIGIT_BITS * r))",
     "np.ldexp(1.0, np.where(e == EZERO, 0, e + 54 - DIGIT_BITS * r))", "sigma trick: 0.75 dropped"),
    ("ozaki", "            lo[i, j] = math.fsum(terms + [-h])\n", "            lo[i, j] = 0.0\n",
     "exact recombination: low word dropped"),
    ("ozaki", "T = 2 * k if mode == \"full\" else k + 1", "T = 2 * k if mode == \"full\" else k",
     "triangular set: last anti-diagonal dropped"),
    ("ozaki", "        v = np.max(np.abs(res), axis=1) if M.shape[1] else np.zeros(M.shape[0])\n",
     "        v = np.max(np.abs(M), axis=1) if M.shape[1] else np.zeros(M.shape[0])\n",
     "adaptive slicing: no rescan of the residual"),
    ("ozaki", "0.75 * np.ldexp(1.0, np.where(e == EZERO, 0, e + alpha)))",
     "0.75 * np.ldexp(1.0, np.where(e == EZERO, 0, e + alpha + 1)))", "adaptive slicing: sigma off by one"),
    ("ozaki", "        res = res - sl\n", "        res = res + sl\n", "adaptive slicing: residual wrong sign"),
    ("refine", "omega = 2.0 * (math.sqrt", "omega = (math.sqrt", "cluster threshold: factor 2 dropped"),
    ("refine", " + p[\"Lam\"] * float(np.linalg.norm(r)))", ")", "cluster threshold: max|lam| ||r|| term dropped"),
    ("refine", "int(np.max(h)), delta * g, opts.k_cap)", "int(np.max(h)), delta, opts.k_cap)",
     "k_W: gap factor dropped"),
    ("refine", "info[\"step\"] > 0.5 * prev_step", "info[\"step\"] > prev_step", "stagnation: growth for failure to halve"),
    ("refine", "if noncontract >= 2:", "if noncontract >= 1:", "stagnation: one failing step stops"),
    ("refine", "/ (xs * g_new) if", "/ (xs) if", "stopping test: gap dropped"),
    ("refine", "g_new, Lam_new = min_gap(lam, omega)", "g_new, Lam_new = min_gap(lam, 0.0)",
     "stopping test: cluster gaps kept"),
    ("refine", "    ql = ql + X1 * Vl\n", "    ql = ql\n", "estimates: low word of V dropped"),
    ("refine", "Res = dd.dd_add(Vh, Vl, -mh, -ml)[0]", "Res = dd.dd_add(Vh, Vl, -mh, 0.0 * ml)[0]",
     "Res: low word of X1 diag(lam) dropped"),
    ("refine", "lam = dd.dd_div_dd(dh, dl, nh, nl)[0]", "lam = dh / nh", "estimates: FP64 division"),
    ("refine", "Up = oz.ozaki_product(X1, E, kU, kU, kU + 1,", "Up = oz.ozaki_product(X1, E, kU, kU, kU,",
     "U: last anti-diagonal dropped"),
    ("refine", "Wp = oz.ozaki_product(X1.T, Res, min(sX, kW), kW, kW + 1,",
     "Wp = oz.ozaki_product(X1.T, Res, min(sX, kW), kW, kW,", "W: last anti-diagonal dropped"),
    ("refine", "V = oz.ozaki_product(A, X1, kV, sX, kV + 1,", "V = oz.ozaki_product(A, X1, kV, sX, kV,",
     "V: last anti-diagonal dropped"),
    ("ozaki", "    return row_exponents(M.T)\n", "    return row_exponents(M)\n", "column exponents: row maxima taken"),
    ("ozaki", "0.75 * np.ldexp(1.0, np.where(f == EZERO, 0, f + beta)))",
     "np.ldexp(1.0, np.where(f == EZERO, 0, f + beta)))", "tau: 0.75 dropped"),
    ("ozaki", "T = 2 * k if mode == \"full\" else k + 1", "T = 2 * k - 1 if mode == \"full\" else k + 1",
     "full pair set: last pair dropped"),
    ("ozaki", "ceil_log2(np.max(np.abs(M), axis=1)) if", "ceil_log2(np.max(np.abs(M), axis=0)) if",
     "row exponents: column maxima taken"),
    ("ddarith", "_SPLITTER = 134217729.0", "_SPLITTER = 67108865.0", "Veltkamp split: 2^26 + 1"),
    ("ddarith", "    se = se + te\n", "    se = se\n", "dd add: low words' rounding error dropped"),
    ("ddarith", "    se = se + th\n", "    se = se\n", "dd add: low words' sum dropped"),
    ("ddarith", "            e = e + a * Rl[k:k + 1, :]\n", "            e = e\n", "dd matmul: low words of R dropped"),
    ("ddarith", "sl = sl + (t + e)", "sl = sl + t", "dd matmul: product error dropped"),
    ("ddarith", "ph, pl = dd_mul_d(bh, bl, q1)", "ph, pl = dd_mul_d(bh, 0.0 * bl, q1)",
     "dd division: low word of the divisor dropped"),
    ("ddarith", "    lo = a - hi\n", "    lo = a + hi\n", "split: low part wrong sign"),
    ("refine", "return int(min(max(b, 3), 47))", "return int(min(max(b, 3), 53))", "beta: clamp at 53"),
    ("refine", "    return ex - 1\n\n\ndef ceil_log2f", "    return ex\n\n\ndef ceil_log2f", "floor log2: off by one"),
    ("refine", "            return k\n    return k_cap\n", "            return k\n    return k_cap - 1\n",
     "slice rule: one plane below the cap"),
    ("refine", "eAmax = int(np.max(eA))", "eAmax = int(np.min(eA))", "k_V: smallest row exponent of A"),
    ("refine", "fmax = int(np.max(f))", "fmax = int(np.min(f))", "k_V: smallest column exponent of X"),
    ("refine", "kW = slices_for(n, int(np.max(f)), int(np.max(h))", "kW = slices_for(n, int(np.max(f)), int(np.min(h))",
     "k_W: smallest column exponent of Res"),
    ("truth", "        diff = lam[None, :] - lam[:, None]\n", "        diff = lam[:, None] - lam[None, :]\n",
     "reference eigenvectors: gap of wrong sign"),
    ("truth", "np.fill_diagonal(E, (rd_h + rd_l) / 2.0)", "np.fill_diagonal(E, (rd_h + rd_l))",
     "reference eigenvectors: r_ii not halved"),
    ("truth", "nh, nl = dd.dd_add(Sh, Sl, ph, pl)", "nh, nl = dd.dd_add(Sh, Sl, -ph, -pl)",
     "reference eigenvectors: s_ij - lam_j r_ij"),
    ("truth", "Gh, Gl = dd.dd_matmul(Xh.T, Xl.T, Xh, Xl)", "Gh, Gl = dd.dd_matmul(Xh.T, None, Xh, None)",
     "reference eigenvectors: X^T X without low words"),
    ("truth", "Vh, Vl = dd.dd_matmul(A, None, Xh, Xl)", "Vh, Vl = dd.dd_matmul(A, None, Xh, None)",
     "reference eigenvectors: A X without the low word"),
    ("truth", "    s[s == 0] = 1.0\n", "    s[s == 0] = 0.0\n", "forward error: orthogonal columns zeroed"),
    ("truth", "P = Qh - Qt @ (Qt.T @ Qh)", "P = Qh - Qh @ (Qt.T @ Qh)", "subspace error: wrong basis in the projector"),
]


def _mutant_package(module, old, new):
    name = "oracle_mutant"
    pkg = types.ModuleType(name)
    pkg.__path__ = []
    saved = {k: sys.modules.get(k) for k in [name] + [f"{name}.{m}" for m in MODULES]}
    sys.modules[name] = pkg
    try:
        for m in MODULES:
            path = os.path.join(ROOT, "oracle", m + ".py")
            src = open(path).read()
            if m == module:
                assert src.count(old) == 1, (m, old)
                src = src.replace(old, new)
            mod = types.ModuleType(f"{name}.{m}")
            mod.__package__ = name
            mod.__file__ = path
            sys.modules[mod.__name__] = mod
            exec(compile(src, path, "exec"), mod.__dict__)
            setattr(pkg, m, mod)
    finally:
        for k, v in saved.items():
            if v is None:
                sys.modules.pop(k, None)
            else:
                sys.modules[k] = v
    return pkg


def _pins():
    """Every pin as a zero-argument call, cheapest first."""
    calls = []
    for mod in (tdd, toz, trf):
        for nm in sorted(dir(mod)):
            fn = getattr(mod, nm)
            if not nm.startswith("test_") or not callable(fn) or nm == "test_golden_workload0_regression":
                continue
            marks = getattr(fn, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            if not params:
                calls.append((f"{mod.__name__}.{nm}", fn, {}))
                continue
            argnames, values = params[0].args
            names = [a.strip() for a in argnames.split(",")]
            for v in values:
                kw = dict(zip(names, v)) if len(names) > 1 else {names[0]: v}
                calls.append((f"{mod.__name__}.{nm}{list(kw.values())}", fn, kw))
    return calls


def _outcome(fn, kw):
    """None if the pin passes (or skips), "assert" if one of its checks fails, else the name
    of the exception that stopped it (a crash, e.g. a shape error on a transposed operand)."""
    try:
        fn(**kw)
    except pytest.skip.Exception:
        return None
    except AssertionError:
        return "assert"
    except Exception as e:
        return type(e).__name__
    return None


def test_every_snippet_is_in_the_oracle():
    for module, old, _, what in MUTANTS:
        src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
        assert src.count(old) == 1, what


def test_unchanged_copy_passes_every_pin(monkeypatch):
    # the control: an unchanged copy fails no pin, so a failure below is the planted mistake's
    pkg = _mutant_package(None, None, None)
    _patch(monkeypatch, pkg)
    failed = [(nm, o) for nm, fn, kw in _pins() if (o := _outcome(fn, kw)) is not None]
    assert failed == []


def _patch(monkeypatch, pkg):
    monkeypatch.setattr(tdd, "dd", pkg.ddarith)
    monkeypatch.setattr(toz, "oz", pkg.ozaki)
    for attr, m in (("dd", pkg.ddarith), ("oz", pkg.ozaki), ("rf", pkg.refine), ("tr", pkg.truth)):
        monkeypatch.setattr(trf, attr, m)


@pytest.mark.parametrize("module,old,new,what", MUTANTS, ids=[m[3] for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, module, old, new, what):
    pkg = _mutant_package(module, old, new)
    _patch(monkeypatch, pkg)
    # a pin must reject the copy through one of its checks; a copy that only makes some pins
    # crash (a shape error, an exhausted search) does not count as caught
    crashes = []
    for nm, fn, kw in _pins():
        o = _outcome(fn, kw)
        if o == "assert":
            return
        if o is not None:
            crashes.append((nm, o))
    pytest.fail(f"no pin check catches: {what} (crashes: {crashes[:3]})")
