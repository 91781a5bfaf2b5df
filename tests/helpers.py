"""Small shared helpers for the tests (input construction and error norms only)."""
import numpy as np

import synth


def rel_fro(a, b):
    """||a - b||_F / ||b||_F."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def small_system(n, n_v, n_c, n_mu=None, seed_index=50, n_pw=None):
    """A small seeded system; `n` an int or (n1, n2, n3).  With n_mu None the
    points are all QRCP pivots up to min(N_r, 2 * pairs)."""
    if isinstance(n, int):
        n = (n, n, n)
    n = tuple(int(v) for v in n)
    n_r = int(np.prod(n))
    n_e = n_v + n_c
    if n_pw is None:
        n_pw = min(max(2 * n_e, 24), n_r - 8)
    phi = synth.make_orbitals(n, n_e, 1000 + seed_index, n_pw=n_pw)
    energies = synth.make_energies(n_v, n_c, 2000 + seed_index)
    if n_mu is None:
        n_mu = min(n_r, 2 * n_v * n_c)
    mu = synth.qrcp_points(phi, n_v, n_mu)
    cell = tuple(v * synth.GRID_SPACING_BOHR for v in n)
    return synth.System(n=n, cell=cell, n_v=n_v, n_c=n_c, phi=phi, energies=energies,
                        mu_idx=mu, name=f"small{n}")


# ------------------------------------------------------------ golden fixtures

GOLDEN_DIR = __import__("pathlib").Path(__file__).resolve().parent / "golden"


def load_golden(name):
    """`key: value` lines of tests/golden/<name> ('#' starts a comment)."""
    out = {}
    for line in (GOLDEN_DIR / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if line:
            key, val = line.split(":", 1)
            out[key.strip()] = val.strip()
    return out


def eval_expr(text, **names):
    """Evaluate an arithmetic expression of a fixture: numbers, + - * / **,
    parentheses, pi and the given names, nothing else."""
    import ast
    import math
    import operator

    ops = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul, ast.Div: operator.truediv,
           ast.Pow: operator.pow, ast.USub: operator.neg, ast.UAdd: operator.pos}
    env = dict(pi=math.pi, **names)

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
            return float(node.value)
        if isinstance(node, ast.Name) and node.id in env:
            return float(env[node.id])
        if isinstance(node, ast.BinOp) and type(node.op) in ops:
            return ops[type(node.op)](ev(node.left), ev(node.right))
        if isinstance(node, ast.UnaryOp) and type(node.op) in ops:
            return ops[type(node.op)](ev(node.operand))
        raise ValueError(f"unsupported expression element: {ast.dump(node)}")

    return ev(ast.parse(text, mode="eval"))


def plane_wave_golden(n_mu):
    """The worked example of tests/golden/plane_wave_two_pairs.txt: a System
    with N_v = 1, N_c = 2 and n_mu QRCP points, the unit pair directions u
    (N_r x 2) and the fixture itself."""
    g = load_golden("plane_wave_two_pairs.txt")
    n = tuple(int(v) for v in g["grid"].split())
    h = float(g["spacing_bohr"])
    n_r = int(np.prod(n))
    z, y, x = np.meshgrid(*(np.arange(k) for k in n[::-1]), indexing="ij")  # x fastest
    coords = (x.reshape(-1), y.reshape(-1), z.reshape(-1))

    def phase(mode):
        m = [int(v) for v in g[f"mode {mode}"].split()]
        return 2 * np.pi * sum(mi * ci / ni for mi, ci, ni in zip(m, coords, n))

    phi = np.empty((n_r, 3), order="F")
    phi[:, 0] = 1 / np.sqrt(n_r)
    phi[:, 1] = np.sqrt(2 / n_r) * np.cos(phase("c1"))
    phi[:, 2] = np.sqrt(2 / n_r) * np.sin(phase("c2"))
    energies = np.array([float(g["energy v"]), float(g["energy c1"]), float(g["energy c2"])])
    mu = synth.qrcp_points(phi, 1, n_mu)
    s = synth.System(n=n, cell=tuple(k * h for k in n), n_v=1, n_c=2, phi=phi, energies=energies,
                     mu_idx=mu, name="plane_wave_two_pairs")
    u = phi[:, 1:3] * np.sqrt(n_r)  # pair directions: v .* c_i = u_i / sqrt(N_r)
    u /= np.linalg.norm(u, axis=0)
    return s, u, g


def plane_wave_golden_eps_inv(u, g, x, w):
    """eps^-1 X from the fixture's closed-form eigenvalues at frequency w."""
    lam = np.array([eval_expr(g["lambda c1"], w=w), eval_expr(g["lambda c2"], w=w)])
    return x + u @ ((1 / lam - 1)[:, None] * (u.T @ x))
