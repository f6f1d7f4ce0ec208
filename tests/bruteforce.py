"""Brute-force and closed-form checkers used to pin the oracle.

Written from the definitions only (arXiv 2302.10083, Section 2): a cube is an
implicant when every minterm it covers is in the support I = ON u DC; it is
prime when no one-digit extension (a 0/1 digit turned into *) is an implicant.
Nothing here runs Merge or Reduce.
"""
from __future__ import annotations

import itertools
from math import comb, factorial

import numpy as np


def digits(n: int) -> np.ndarray:
    """(3^n, n) array: digit i of every rho (digit i is variable x_{i+1})."""
    r = np.arange(3 ** n, dtype=np.int64)
    out = np.empty((3 ** n, n), dtype=np.int8)
    for i in range(n):
        out[:, i] = r % 3
        r //= 3
    return out


def mask_value(n: int):
    """(mask, value) of every cube, int64 arrays indexed by rho."""
    d = digits(n)
    w = (1 << np.arange(n, dtype=np.int64))
    mask = ((d != 2) * w).sum(axis=1) if n else np.zeros(1, dtype=np.int64)
    value = ((d == 1) * w).sum(axis=1) if n else np.zeros(1, dtype=np.int64)
    return mask.astype(np.int64), value.astype(np.int64)


def implicants(n: int, support: np.ndarray) -> np.ndarray:
    """Bool array over rho: every covered minterm x has support[x]."""
    mask, value = mask_value(n)
    off = np.nonzero(~np.asarray(support, dtype=bool))[0].astype(np.int64)
    imp = np.ones(3 ** n, dtype=bool)
    if off.size == 0:
        return imp
    step = max(1, 4_000_000 // max(off.size, 1))
    for s in range(0, 3 ** n, step):
        m = mask[s:s + step, None]
        v = value[s:s + step, None]
        imp[s:s + step] = ~np.any((off[None, :] & m) == v, axis=1)
    return imp


def primes_from_implicants(n: int, imp: np.ndarray) -> np.ndarray:
    """Implicants with no implicant one-digit extension."""
    d = digits(n)
    prime = imp.copy()
    rho = np.arange(3 ** n, dtype=np.int64)
    for i in range(n):
        binary = d[:, i] != 2
        ext = rho + (2 - d[:, i].astype(np.int64)) * 3 ** i
        prime &= ~(binary & imp[np.where(binary, ext, rho)])
    return prime


def primes(n: int, support: np.ndarray) -> np.ndarray:
    return primes_from_implicants(n, implicants(n, support))


def support_of(n: int, on_bits: np.ndarray, dc_bits: np.ndarray | None = None) -> np.ndarray:
    on = np.unpackbits(on_bits, bitorder="little")[: 1 << n].astype(bool)
    if dc_bits is None:
        return on
    return on | np.unpackbits(dc_bits, bitorder="little")[: 1 << n].astype(bool)


def bitmap_from_bool(cells: np.ndarray) -> np.ndarray:
    return np.packbits(cells.astype(bool), bitorder="little")


def bool_from_bitmap(bitmap: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(np.asarray(bitmap, dtype=np.uint8), bitorder="little")[: 3 ** n].astype(bool)


# ---- symmetric functions --------------------------------------------------

def symmetric_support(n: int, W) -> np.ndarray:
    """Support of the symmetric function that is 1 exactly on Hamming weights in W."""
    x = np.arange(1 << n, dtype=np.int64)
    pop = np.zeros_like(x)
    for i in range(n):
        pop += (x >> i) & 1
    return np.isin(pop, list(W))


def symmetric_prime_cells(n: int, W) -> np.ndarray:
    """Closed form: a cube with a ones, b zeros and w stars is prime iff
    {a..a+w} is inside W, (a = 0 or a-1 not in W) and (b = 0 or a+w+1 not in W)."""
    W = set(W)
    d = digits(n)
    a = (d == 1).sum(axis=1)
    b = (d == 0).sum(axis=1)
    w = (d == 2).sum(axis=1)
    out = np.zeros(3 ** n, dtype=bool)
    for aa in range(n + 1):
        for ww in range(n + 1 - aa):
            bb = n - aa - ww
            ok = all(k in W for k in range(aa, aa + ww + 1))
            ok = ok and (aa == 0 or (aa - 1) not in W) and (bb == 0 or (aa + ww + 1) not in W)
            if ok:
                out |= (a == aa) & (w == ww) & (b == bb)
    return out


def symmetric_prime_count(n: int, W) -> int:
    W = set(W)
    total = 0
    for aa in range(n + 1):
        for ww in range(n + 1 - aa):
            bb = n - aa - ww
            ok = all(k in W for k in range(aa, aa + ww + 1))
            ok = ok and (aa == 0 or (aa - 1) not in W) and (bb == 0 or (aa + ww + 1) not in W)
            if ok:
                total += factorial(n) // (factorial(aa) * factorial(bb) * factorial(ww))
    return total


# ---- expectations for i.i.d. Bernoulli(p) support ---------------------------

def rho_positive(n: int, m: int) -> int:
    """rho of the positive term of point m: digit i is 1 where m has x_i, else *."""
    return sum((1 if (m >> i) & 1 else 2) * 3 ** i for i in range(n))


def monotone_case(n: int, seed: int):
    """A monotone function with no symmetry (an OR of 3n random positive
    terms) as a support array, and its minimal true points in ascending rho
    of their positive terms."""
    rng = np.random.default_rng(seed)
    t = np.arange(1 << n)
    sup = np.zeros(1 << n, dtype=bool)
    for _ in range(3 * n):
        size = int(rng.integers(1, max(2, n // 2) + 1))
        T = int(np.bitwise_or.reduce(1 << rng.choice(n, size=size, replace=False)))
        sup |= (t & T) == T
    minimal = sup.copy()
    for i in range(n):
        has = ((t >> i) & 1) == 1
        minimal &= ~(has & sup[t ^ (1 << i)])
    return sup, sorted(t[minimal].tolist(), key=lambda m: rho_positive(n, m))


def rho_of_pair(n: int, mask: int, value: int) -> int:
    """rho of the cube whose (mask, value) pair is given: digit i is * where
    mask has no bit i, else value's bit i."""
    return sum(((value >> i) & 1 if (mask >> i) & 1 else 2) * 3 ** i for i in range(n))


def unate_case(n: int, seed: int, nu: int):
    """The monotone function of monotone_case with the inputs in nu negated,
    g(x) = f(x xor nu), as a support array, and its primes in closed form as
    (mask, value) pairs in ascending rho: minimal true point m of f gives the
    cube with literal x_i = 1 xor nu_i for i in m, * elsewhere."""
    sup, mins = monotone_case(n, seed)
    t = np.arange(1 << n)
    pairs = sorted(((m, m & ~nu & ((1 << n) - 1)) for m in mins), key=lambda p: rho_of_pair(n, *p))
    return sup[t ^ nu], pairs


def expected_implicants(n: int, p: float) -> float:
    return sum(comb(n, w) * 2 ** (n - w) * p ** (2 ** w) for w in range(n + 1))


def expected_primes(n: int, p: float) -> float:
    """A cube with w stars is prime iff its 2^w minterms are in I and, for each of
    its n-w binary digits, the 2^w minterms of the sibling cube are not all in I;
    the n-w sibling cubes and the cube are disjoint, so the events are independent."""
    return sum(comb(n, w) * 2 ** (n - w) * p ** (2 ** w) * (1 - p ** (2 ** w)) ** (n - w)
               for w in range(n + 1))


def cube_string(n: int, rho: int) -> str:
    s = []
    for _ in range(n):
        s.append("01*"[rho % 3])
        rho //= 3
    return "".join(s)


def rho_of_string(s: str) -> int:
    return sum("01*".index(ch) * 3 ** i for i, ch in enumerate(s))


def all_functions(n: int):
    """Every truth table of n variables as a bool array."""
    m = 1 << n
    for f in range(1 << m):
        yield f, np.array([(f >> t) & 1 for t in range(m)], dtype=bool)


def perm_digits(n: int, perm) -> np.ndarray:
    """Index map: new_rho[rho] for the cube whose digit perm[i] is old digit i."""
    d = digits(n)
    nd = np.empty_like(d)
    for i, j in enumerate(perm):
        nd[:, j] = d[:, i]
    return (nd.astype(np.int64) * (3 ** np.arange(n, dtype=np.int64))).sum(axis=1)


def load_golden(path: str):
    rows, meta = [], {}
    for line in open(path):
        line = line.strip()
        if not line:
            continue
        if line.startswith("#"):
            body = line[1:].strip()
            if body.startswith("n="):
                for tok in body.split():
                    k, v = tok.split("=")
                    meta[k] = v
            continue
        cube, rho, mask, value = line.split()
        rows.append((cube, int(rho), int(mask), int(value)))
    return meta, rows


__all__ = [name for name in dir() if not name.startswith("_")] + ["itertools"]
