"""Plant one plausible mistake at a time in a scratch copy of the oracle and
check that the CPU pins (``pytest -m "not gpu"``) catch it.

On demand only (about 15 minutes; pytest does not collect this file):

    python tests/plant_oracle_mistakes.py            # every mistake
    python tests/plant_oracle_mistakes.py 3 7        # the 4th and the 8th

Each entry names the oracle file, the exact text replaced, its replacement
and a label.  The repository itself is never modified: the oracle, the
tests and their inputs are copied to a temporary directory per mistake.
Exit status 1 when a mistake is missed.
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTS = [
 ("qtt.py", "A = rest.reshape((m, -1), order='F')          # unfolding m_k x n_k", "A = rest.reshape((m, -1), order='C')          # unfolding m_k x n_k", "tt_svd C-order unfolding"),
 ("qtt.py", "tau = (eps / np.sqrt(d - 1)) * np.linalg.norm(v) if d > 1 else 0.0", "tau = (eps / np.sqrt(d)) * np.linalg.norm(v) if d > 1 else 0.0", "tt_svd threshold sqrt(d)"),
 ("qtt.py", "tau = (eps / np.sqrt(d - 1)) * np.linalg.norm(v) if d > 1 else 0.0", "tau = eps * np.linalg.norm(v) if d > 1 else 0.0", "tt_svd threshold eps*||A|| per step"),
 ("qtt.py", "        if s[k - 1] > 0 and s[k] / s[k - 1] < delta:\n            r = k\n            break", "        if s[k - 1] > 0 and s[k] / s[k - 1] < delta:\n            r = k + 1\n            break", "drop_rank off by one"),
 ("qtt.py", "            modes.append((0, b))\n            if b < dy:\n                modes.append((1, b))", "            modes.append((0, b))\n            if b < dy:\n                modes.insert(len(modes) - 1, (1, b))", "mode_map y before x"),
 ("conv.py", "    s = np.sinc(B * m * h)", "    s = np.sinc(B * m * h / np.pi)", "sinc convention"),
 ("conv.py", "        A = 1.0 / (h * s.sum())", "        A = 1.0 / s.sum()", "normalisation without h"),
 ("toeplitz.py", "    Y = np.einsum('pjiq,aib->pajqb', O, X)", "    Y = np.einsum('pijq,aib->pajqb', O, X)", "matvec transposed operator"),
 ("rsvd.py", "        if min(m, n) <= rmax + p:", "        if min(m, n) < rmax + p:", "rsvd fallback boundary"),
 ("rsvd.py", "    B = Q.conj().T @ A", "    B = Q.T @ A", "rsvd missing conj"),
 ("qfft.py", "t = np.exp(sgn * 2j * np.pi * i * 2.0 ** (kk - 1) / 2.0 ** p) if c else 1.0", "t = np.exp(sgn * 2j * np.pi * i * 2.0 ** kk / 2.0 ** p) if c else 1.0", "qfft twiddle exponent"),
 ("qfft.py", "    sgn = 1.0 if inverse else -1.0", "    sgn = -1.0 if inverse else 1.0", "qfft sign convention"),
 ("qfft.py", "        g[j] = taps[c + j - h]", "        g[j] = taps[c + j + h]", "padded kernel offset"),
 ("qfft.py", "    h = (N - 1) // 2\n    Ic = np.asarray(Ic)", "    h = (N + 1) // 2\n    Ic = np.asarray(Ic)", "linear_part shift"),
 ("qfft.py", "    return [np.transpose(c, (2, 1, 0)).copy() for c in reversed(cores)]", "    return [np.transpose(c, (0, 1, 2)).copy() for c in reversed(cores)]", "reverse without bond swap"),
 ("qtt.py", "        P = np.einsum('aib,ac,cid->bd', np.conj(c), P, c)", "        P = np.einsum('aib,ac,cid->bd', c, P, c)", "norm without conj"),
 ("qtt.py", "    for k in range(d - 1, 0, -1):\n        r0, _, r1 = cores[k].shape", "    for k in range(0):\n        r0, _, r1 = cores[k].shape", "tt_round without orthogonalisation"),
 ("rsvd.py", "        cores.append(U[:, :r].reshape((r_prev, 2, r), order='F'))\n        rest = s[:r, None] * Vh[:r, :]", "        cores.append(U[:, :r].reshape((r_prev, 2, r), order='F'))\n        rest = Vh[:r, :]", "tt_rsvd drops Sigma"),
 ("qfft.py", "        z = np.einsum('aib,cid->acibd', a, b)", "        z = np.einsum('aib,cid->acibd', a, np.conj(b))", "hadamard conj"),
 ("qfft.py", "        elif lo < k < hi:\n            O = np.zeros((2, 2, 2, 2), dtype=np.complex128)\n            for c in range(2):\n                O[c, 0, 0, c] = O[c, 1, 1, c] = 1.0", "        elif lo < k < hi:\n            O = np.zeros((2, 2, 2, 2), dtype=np.complex128)\n            for c in range(2):\n                O[c, 0, 0, 0] = O[c, 1, 1, 0] = 1.0", "pass-through drops the branch"),
 ("qfft.py", "        Y[0] = Y[0] / 2.0 ** d", "        Y[0] = Y[0] / 2.0 ** (d - 1)", "inverse scaling"),
 ("pipeline.py", "        gk = np.einsum('lir,la,br->aib', W, np.conj(Lp), np.conj(Rp))", "        gk = np.einsum('lir,la,br->aib', W, Lp, np.conj(Rp))", "core_grads missing conj"),
]


def run(f, a, b, name):
    tmp = tempfile.mkdtemp(prefix="plant_")
    try:
        for item in ("oracle", "synth", "tests", "paper_2301_13339_gb300", "bench.py",
                     "__graft_entry__.py", "include"):
            src = os.path.join(ROOT, item)
            dst = os.path.join(tmp, item)
            if os.path.isdir(src):
                shutil.copytree(src, dst, ignore=shutil.ignore_patterns("__pycache__", "obj"))
            else:
                shutil.copy(src, dst)
        p = os.path.join(tmp, "oracle", f)
        s = open(p).read()
        if a not in s:
            return name, "pattern not found"
        open(p, "w").write(s.replace(a, b, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-q", "-x", "-m", "not gpu",
                            "-p", "no:cacheprovider", "--ignore=tests/test_abi_symbols.py",
                            "--ignore=tests/test_multirank_cpu.py",
                            "--ignore=tests/test_partitioned_tt_svd_cpu.py"],
                           cwd=tmp, capture_output=True, text=True, timeout=1800)
        first = next((ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")), "")
        return name, ("caught  " + first) if r.returncode != 0 else "MISSED"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def main(argv):
    sel = set(argv)
    missed = 0
    for i, (f, a, b, name) in enumerate(MUTS):
        if sel and str(i) not in sel:
            continue
        label, verdict = run(f, a, b, name)
        missed += not verdict.startswith("caught")
        print(f"{i:2d} {label:40s} {verdict}", flush=True)
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
