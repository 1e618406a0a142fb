"""Planted mistakes in the CPU oracle must fail its pins.

Each mutant rewrites one site of an oracle module's source: a dropped term, a wrong sign,
an index off by one, a transposed operand or a wrong constant. The rewritten module is
loaded in place of the original for the length of one test, and the pin battery of
tests/test_oracle_*.py is run against it: at least one pin must fail. The battery runs the
pins that call the mutated module directly first and stops at the first failure. The
unmutated oracle passes the same battery through the same harness
(test_battery_passes_unmutated), so a mutant's failure comes from the mutation.

Only mutants that change a result are listed. Mutants that leave every result unchanged
are not: for example, Algorithm 1's a_j taken against f_j + f_{j-1} instead of f_j
(q_j . f_{j-1} = 0 by construction), or the sign of 2 pi J_a in the Lieb-Wu equations
(the centred J set and its mirror image give the same energy). The GPU library is not
involved; everything runs on the CPU.
"""
import importlib
import inspect
import signal
import sys
import types
import warnings
from dataclasses import dataclass

import numpy as np
import pytest

import oracle
import test_oracle_complex
import test_oracle_mlp
import test_oracle_observables
import test_oracle_pins

ORACLE_MODULES = ("basis", "hamiltonian", "tridiag", "lanczos", "dense", "observables",
                  "complex_hopping", "mlp", "bethe")
PIN_MODULES = (test_oracle_pins, test_oracle_complex, test_oracle_observables, test_oracle_mlp)
CASE_SECONDS = 30   # a pin case that runs longer than this under a mutant counts as failed


# ------------------------------------------------------------------------ the pin battery
def _expand(fn):
    """The keyword sets of a test function's stacked parametrize marks (one empty set when
    it has none)."""
    grid = [{}]
    for mark in getattr(fn, "pytestmark", []):
        if mark.name != "parametrize":
            continue
        names, values = mark.args[0], mark.args[1]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        rows = []
        for v in values:
            if hasattr(v, "marks") and hasattr(v, "values"):   # pytest.param(...)
                v = v.values if len(names) > 1 else v.values[0]
            rows.append(dict(zip(names, v if len(names) > 1 else (v,))))
        grid = [dict(g, **r) for r in rows for g in grid]
    return grid


def _battery():
    cases = []
    for mod in PIN_MODULES:
        for name, fn in vars(mod).items():
            if not (name.startswith("test_") and inspect.isfunction(fn)):
                continue
            params = set(inspect.signature(fn).parameters)
            for kw in _expand(fn):
                assert set(kw) == params, f"{mod.__name__}.{name} takes fixtures"
                cases.append((f"{mod.__name__}.{name}{sorted(kw.items())!r}"[:160], fn, kw))
    return cases


BATTERY = _battery()


class _CaseTimeout(Exception):
    pass


def _on_alarm(signum, frame):
    raise _CaseTimeout()


def _ordered(name):
    """The battery with the cases that call oracle.<name> directly first (they usually
    fail first under a mutant of that module), then the rest in file order."""
    orig = importlib.import_module("oracle." + name)
    first, rest = [], []
    for case in BATTERY:
        fn = case[1]
        aliases = [a for a, v in vars(sys.modules[fn.__module__]).items() if v is orig]
        src = inspect.getsource(fn)
        (first if any(a + "." in src for a in aliases) else rest).append(case)
    return first + rest


def _first_failure(cases):
    """Run the cases; return (case id, error) of the first that fails, or None."""
    old = signal.signal(signal.SIGALRM, _on_alarm)
    try:
        for cid, fn, kw in cases:
            signal.setitimer(signal.ITIMER_REAL, CASE_SECONDS)
            try:
                with warnings.catch_warnings(), np.errstate(all="ignore"):
                    warnings.simplefilter("ignore")
                    fn(**kw)
            except _CaseTimeout:
                return cid, "timed out"
            except Exception as e:   # an assertion or any error counts as a failed pin
                return cid, f"{type(e).__name__}: {e}"[:200]
            finally:
                signal.setitimer(signal.ITIMER_REAL, 0)
        return None
    finally:
        signal.signal(signal.SIGALRM, old)


# ------------------------------------------------------------------------------ mutants
@dataclass
class Mutant:
    id: str
    module: str
    edits: tuple   # (old, new, occurrence): replace the occurrence-th (1-based) copy of old


def M(id, module, *edits):
    return Mutant(id, module, tuple(e if len(e) == 3 else (e[0], e[1], 1) for e in edits))


MUTANTS = [
    # basis: Sec. 2.1, Eq. 2
    M("popcount-drops-top-byte", "basis", ("for k in range(8):", "for k in range(7):")),
    M("states-descending", "basis", ("sorted(vals)", "sorted(vals, reverse=True)")),
    M("states-skip-last-site", "basis",
      ("combinations(range(n_sites), n_particles)", "combinations(range(n_sites - 1), n_particles)")),
    M("rank-off-by-one", "basis", ("r = np.searchsorted(states, s)", "r = np.searchsorted(states, s) - 1")),
    M("dimension-uses-n-up-twice", "basis",
      ("len(species_states(n_sites, n_dn))", "len(species_states(n_sites, n_up))")),
    # hamiltonian: Eq. 1 plus the on-site term, fermion signs
    M("sign-mask-includes-low-end", "hamiltonian", ("~((1 << (lo + 1)) - 1)", "~((1 << lo) - 1)")),
    M("sign-mask-includes-high-end", "hamiltonian", ("((1 << hi) - 1) &", "((1 << (hi + 1)) - 1) &")),
    M("fermion-sign-dropped", "hamiltonian",
      ("sign = np.where(npass % 2 == 0, 1.0, -1.0)", "sign = np.ones(len(src))")),
    M("fermion-sign-inverted", "hamiltonian",
      ("sign = np.where(npass % 2 == 0, 1.0, -1.0)", "sign = np.where(npass % 2 == 0, -1.0, 1.0)")),
    M("hop-sign-up-species", "hamiltonian",
      ("rows.append(tgt); cols.append(src); vals.append(-t * sign)",
       "rows.append(tgt); cols.append(src); vals.append(t * sign)", 1)),
    M("hop-sign-down-species", "hamiltonian",
      ("rows.append(tgt); cols.append(src); vals.append(-t * sign)",
       "rows.append(tgt); cols.append(src); vals.append(t * sign)", 2)),
    M("down-hop-keeps-wrong-up-rank", "hamiltonian",
      ("tgt = (src // dim_dn) * dim_dn + rank_of(dn, s2)",
       "tgt = (src % len(up)) * dim_dn + rank_of(dn, s2)")),
    M("up-hop-keeps-wrong-down-rank", "hamiltonian",
      ("tgt = rank_of(up, s2) * dim_dn + (src % dim_dn)",
       "tgt = rank_of(up, s2) * dim_dn + (src // len(up)) % dim_dn")),
    M("interaction-or-not-and", "hamiltonian", ("diag = U * popcount(ub & db)", "diag = U * popcount(ub | db)")),
    M("interaction-dropped", "hamiltonian",
      ("rows.append(g); cols.append(g); vals.append(diag)", "rows.append(g); cols.append(g); vals.append(0 * diag)")),
    M("interaction-counts-up-only", "hamiltonian", ("diag = U * popcount(ub & db)", "diag = U * popcount(ub)")),
    M("rows-diagonal-dropped", "hamiltonian",
      ("y = U * popcount(ub & db).astype(np.float64) * x[rows]", "y = 0.0 * x[rows]")),
    M("rows-up-hop-sign", "hamiltonian",
      ("np.add.at(y, src, -t * sign * x[col])", "np.add.at(y, src, t * sign * x[col])", 1)),
    M("rows-down-hop-column", "hamiltonian",
      ("col = (rows[src] // dim_dn) * dim_dn + rank_of(dn, s2)\n        np.add.at(y, src, -t",
       "col = (rows[src] // dim_dn) * dim_dn + (rows[src] % dim_dn)\n        np.add.at(y, src, -t")),
    M("abs-rows-signed-U", "hamiltonian", ("y = abs(U) * popcount", "y = U * popcount")),
    M("abs-rows-down-hops-dropped", "hamiltonian",
      ("np.add.at(y, src, abs(t) * ax[col])", "np.add.at(y, src, 0.0 * ax[col])", 2)),
    M("hop-table-sign-dropped", "hamiltonian", ("lists[r].append((t_, int(sg)))", "lists[r].append((t_, 1))")),
    M("hop-table-source-as-target", "hamiltonian", ("lists[r].append((t_, int(sg)))", "lists[r].append((r, int(sg)))")),
    M("hop-table-bond-order-reversed", "hamiltonian",
      ("for src, s2, sign in hops_of(states, bonds):", "for src, s2, sign in hops_of(states, np.asarray(bonds)[::-1]):")),
    # tridiag: Sturm count and bisection for lambda_min(T), Sec. 2.2
    M("sturm-offdiag-not-squared", "tridiag", ("off = b[i - 1] * b[i - 1] / d", "off = b[i - 1] / d")),
    M("sturm-offdiag-sign", "tridiag", ("d = (a[i] - x) - off", "d = (a[i] - x) + off")),
    M("sturm-offdiag-index", "tridiag", ("off = b[i - 1] * b[i - 1] / d", "off = b[i % len(b)] * b[i % len(b)] / d")),
    M("sturm-last-pivot-skipped", "tridiag", ("for i in range(len(a)):", "for i in range(len(a) - 1):")),
    M("gershgorin-one-side", "tridiag", ("rad[1:] += np.abs(b)", "rad[1:] += 0.0")),
    M("bisection-second-eigenvalue", "tridiag", ("if sturm_count(a, b, mid) >= 1:", "if sturm_count(a, b, mid) >= 2:")),
    # lanczos: Algorithm 1
    M("lanczos-drops-b-f-prev", "lanczos", ("q = matvec(f) - b * f_prev", "q = matvec(f)")),
    M("lanczos-adds-b-f-prev", "lanczos", ("q = matvec(f) - b * f_prev", "q = matvec(f) + b * f_prev")),
    M("lanczos-adds-a-f", "lanczos", ("q = q - a * f", "q = q + a * f")),
    M("lanczos-beta-squared", "lanczos", ("b_next = float(np.sqrt(q @ q))", "b_next = float(q @ q)")),
    M("lanczos-beta-lags", "lanczos", ("E0 = lowest_eigenvalue(res.alpha, res.beta[:-1])",
                                       "E0 = lowest_eigenvalue(res.alpha, [b] + res.beta[:-2])")),
    M("lanczos-loose-stop", "lanczos", ("<= tol * max(abs(E0), 1.0)", "<= 1e5 * tol * max(abs(E0), 1.0)")),
    M("lanczos-early-breakdown", "lanczos", ("BREAKDOWN_REL = 1e-13", "BREAKDOWN_REL = 1e-2")),
    M("lanczos-start-not-normalised", "lanczos", ("f /= nrm", "f /= 1.0")),
    M("lanczos-fixed-steps-ignored", "lanczos", ("if not fixed_steps and j > 1", "if j > 1")),
    M("start-vector-squared-norm", "lanczos", ("return raw / np.sqrt(raw @ raw)", "return raw / (raw @ raw)")),
    # dense: the plain definition of E0 and the ground state's sign gauge
    M("ground-state-row-not-column", "dense", ("psi = v[:, 0].copy()", "psi = v[0, :].copy()")),
    M("ground-state-gauge-flipped", "dense", ("if psi[k] < 0:", "if psi[k] > 0:")),
    M("ground-state-second-level", "dense", ("return float(w[0]), psi", "return float(w[1]), psi")),
    # observables: double occupancy (the on-site term)
    M("double-occupancy-transposed", "observables",
      ("reshape(len(up), len(dn))", "reshape(len(dn), len(up)).T")),
    M("double-occupancy-not-normalised", "observables", ("/ norm2", "/ 1.0")),
    M("double-occupancy-amplitude-not-squared", "observables", (") ** 2", ").__abs__()")),
    M("double-occupancy-up-twice", "observables", ("occ_up @ p2 @ occ_dn", "occ_up @ p2 @ occ_up[:len(dn)]")),
    M("double-occupancy-site-shift", "observables", ("occ_dn = ((dn >> np.uint32(i))", "occ_dn = ((dn >> np.uint32((i + 1) % n_sites))")),
    # complex_hopping: complex amplitude per bond
    M("complex-conjugate-swapped-matrix", "complex_hopping",
      ("np.where(from_j, -tau[b], -np.conj(tau[b]))", "np.where(from_j, -np.conj(tau[b]), -tau[b])")),
    M("complex-conjugate-swapped-everywhere", "complex_hopping",
      ("np.where(from_j, -tau[b], -np.conj(tau[b]))", "np.where(from_j, -np.conj(tau[b]), -tau[b])"),
      ("np.where(at_j, -np.conj(tau[b]), -tau[b])", "np.where(at_j, -tau[b], -np.conj(tau[b]))"),
      ("h[i, j] += -tau[b]\n        h[j, i] += -np.conj(tau[b])", "h[i, j] += -np.conj(tau[b])\n        h[j, i] += -tau[b]")),
    M("complex-t-dropped", "complex_hopping", ("tau = t * np.asarray(tbond, dtype=np.complex128)\n    up",
                                              "tau = np.asarray(tbond, dtype=np.complex128)\n    up")),
    M("complex-rows-diagonal-dropped", "complex_hopping",
      ("y = U * popcount(ub & db).astype(np.float64) * x[rows]", "y = 0.0 * x[rows]")),
    M("complex-one-body-transposed", "complex_hopping",
      ("h[i, j] += -tau[b]", "h[j, i] += -tau[b]")),
    M("complex-u0-down-count", "complex_hopping", ("e[:n_up].sum() + e[:n_dn].sum()", "2.0 * e[:n_up].sum()")),
    M("real-view-imag-sign", "complex_hopping", ("out[1::2] = w.imag", "out[1::2] = -w.imag")),
    M("complex-rows-up-column", "complex_hopping",
      ("col = rank_of(up, s2) * dim_dn + (rows[src] % dim_dn)", "col = rank_of(up, s2) * dim_dn + (rows[src] // dim_dn) % dim_dn")),
    M("complex-rows-end-test", "complex_hopping", ("j = int(bonds[b, 1])", "j = int(bonds[b, 0])")),
    # mlp: the start-vector network
    M("bf16-round-half-up", "mlp", ("np.uint64(0x7FFF) + lsb", "np.uint64(0x8000)")),
    M("bf16-truncates", "mlp", ("np.uint64(0x7FFF) + lsb", "np.uint64(0)")),
    M("features-down-from-up", "mlp", ("x[:, n_sites + i] = (dn >> i) & 1", "x[:, n_sites + i] = (up >> i) & 1")),
    M("features-U-scale", "mlp", ("bf16_round(np.float32(U / 8.0))", "bf16_round(np.float32(U / 4.0))")),
    M("forward-W2-transposed", "mlp", ("h2 = np.tanh(h1b @ W2 + b2)\n    out = h2 @ W3 + b3\n    return",
                                       "h2 = np.tanh(h1b @ W2.T + b2)\n    out = h2 @ W3 + b3\n    return")),
    M("forward-W1-layout", "mlp", ("W1 = p[o:o + n_in * HIDDEN].reshape(n_in, HIDDEN)",
                                   "W1 = p[o:o + n_in * HIDDEN].reshape(HIDDEN, n_in).T")),
    M("forward-h1-unrounded", "mlp", ("h1b = bf16_round(h1) if round_weights else h1\n    h2 = np.tanh(h1b @ W2 + b2)\n    out = h2 @ W3 + b3\n    return",
                                      "h1b = h1\n    h2 = np.tanh(h1b @ W2 + b2)\n    out = h2 @ W3 + b3\n    return")),
    M("forward-outputs-swapped", "mlp", ("return out[:, 0], out[:, 1], (x, h1, h2)", "return out[:, 1], out[:, 0], (x, h1, h2)")),
    M("predict-sign-inverted", "mlp", ("np.where(z >= 0, 1.0, -1.0)", "np.where(z >= 0, -1.0, 1.0)")),
    M("unpack-b1-offset", "mlp", ("b1 = p[o:o + HIDDEN]; o += HIDDEN\n    W2", "b1 = p[o + 1:o + 1 + HIDDEN]; o += HIDDEN\n    W2")),
    M("unpack-W3-layout", "mlp", ("W3 = p[o:o + HIDDEN * 2].reshape(HIDDEN, 2)", "W3 = p[o:o + HIDDEN * 2].reshape(2, HIDDEN).T")),
    M("param-count-short", "mlp", ("+ HIDDEN * 2 + 2\n", "+ HIDDEN * 2\n")),
    M("features-site-order", "mlp", ("x[:, i] = (up >> i) & 1", "x[:, n_sites - 1 - i] = (up >> i) & 1")),
    M("loss-hidden-W2-transposed", "mlp", ("h2 = np.tanh(h1b @ W2 + b2)\n    out = h2 @ W3 + b3\n    a, z",
                                           "h2 = np.tanh(h1b @ W2.T + b2)\n    out = h2 @ W3 + b3\n    a, z")),
    M("loss-weight-not-squared", "mlp", ("weight_scale * psi * psi", "weight_scale * np.abs(psi)")),
    M("loss-sign-term", "mlp", ("np.logaddexp(0.0, -sg * z)", "np.logaddexp(0.0, sg * z)")),
    M("grad-backprop-W2-not-transposed", "mlp", ("g1 = (g2 @ W2.T)", "g1 = (g2 @ W2)")),
    M("grad-dz-sign", "mlp", ("/ (1.0 + np.exp(sg * z))", "/ (1.0 + np.exp(-sg * z))")),
    M("grad-tanh-derivative", "mlp", ("g2 = (dout @ W3.T) * (1.0 - h2 * h2)", "g2 = (dout @ W3.T) * (1.0 - h2)")),
    # bethe: the Lieb-Wu equations for the periodic ring
    M("bethe-theta-half", "bethe", ("return 2.0 * np.arctan(x)", "return np.arctan(x)")),
    M("bethe-u-scale", "bethe", ("u_target = U / (4.0 * t)", "u_target = U / (2.0 * t)")),
    M("bethe-I-parity", "bethe", ("shift_I = 0.0 if M % 2 == 0 else 0.5", "shift_I = 0.5 if M % 2 == 0 else 0.0")),
    M("bethe-J-parity", "bethe", ("shift_J = 0.0 if (N - M) % 2 == 1 else 0.5", "shift_J = 0.5 if (N - M) % 2 == 1 else 0.0")),
    M("bethe-spin-spin-scale", "bethe",
      ("- _theta((lam[:, None] - lam[None, :]) / (2 * u)).sum(axis=1))",
       "- _theta((lam[:, None] - lam[None, :]) / u).sum(axis=1))")),
    M("bethe-charge-sign", "bethe", ("L * k - 2 * np.pi * I + _theta", "L * k - 2 * np.pi * I - _theta")),
    M("bethe-energy-scale", "bethe", ("-2.0 * t * np.sum(np.cos(k))", "-t * np.sum(np.cos(k))")),
    M("bethe-lowest-spin-only", "bethe", ("cands = range(min(n_up, n_dn) + 1)", "cands = [min(n_up, n_dn)]")),
    M("bethe-numbers-off-centre", "bethe", ("q = np.arange(n, dtype=np.float64) - (n - 1) / 2.0",
                                            "q = np.arange(n, dtype=np.float64) - (n - 1) / 2.0 + 1.0")),
]


def _load_mutant(m: Mutant):
    path = importlib.import_module("oracle." + m.module).__file__
    src = open(path).read()
    for old, new, k in m.edits:
        n = src.count(old)
        assert n >= k, f"mutation site {old!r} found {n} times in oracle/{m.module}.py"
        at = -1
        for _ in range(k):
            at = src.index(old, at + 1)
        src = src[:at] + new + src[at + len(old):]
    mod = types.ModuleType("oracle." + m.module)
    mod.__file__ = path
    mod.__package__ = "oracle"
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


def _install(monkeypatch, name, mutant):
    """Put `mutant` in place of oracle.<name> wherever the oracle package and the pin modules
    hold it: the module itself and every object imported from it by name."""
    orig = importlib.import_module("oracle." + name)
    monkeypatch.setitem(sys.modules, "oracle." + name, mutant)
    monkeypatch.setattr(oracle, name, mutant)
    holders = [importlib.import_module("oracle." + n) for n in ORACLE_MODULES if n != name]
    for h in holders + list(PIN_MODULES):
        for attr, val in list(vars(h).items()):
            if val is orig:
                monkeypatch.setattr(h, attr, mutant)
            elif getattr(val, "__module__", None) == orig.__name__ and \
                    getattr(orig, getattr(val, "__name__", ""), None) is val:
                monkeypatch.setattr(h, attr, getattr(mutant, val.__name__))


def test_battery_passes_unmutated():
    assert len(BATTERY) >= 151
    assert _first_failure(BATTERY) is None


def test_mutant_sites_are_unique_enough():
    """Every planted edit names text that exists in the oracle source (a site that went
    missing after an edit of the oracle would silently test nothing)."""
    for m in MUTANTS:
        _load_mutant(m)
    assert len({m.id for m in MUTANTS}) == len(MUTANTS)


@pytest.mark.parametrize("m", MUTANTS, ids=[m.id for m in MUTANTS])
def test_planted_mistake_fails_a_pin(m, monkeypatch):
    cases = _ordered(m.module)
    _install(monkeypatch, m.module, _load_mutant(m))
    hit = _first_failure(cases)
    assert hit is not None, f"mutant {m.id} of oracle/{m.module}.py passes every pin"
