"""Output lengths and input/seed lengths of the extractors (the parameter layer).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each bound is the paper's theorem written out, in double precision, with the
floor taken last.  Error is passed as ``log2_eps = log2(epsilon) < 0`` so that
epsilon = 10^-100 and smaller stay representable.  ``n1`` is the number of input
bits an extraction call takes (the ``n`` of the Toeplitz and Dodis et al.
calls, the ``n - 1`` input bits of Def. ext-circ for Circulant).

Models and adversaries:

* ``seeded``  -- a perfect seed, k2 = n2;
* ``product`` -- two independent weak sources (Thm. 2-weak-source for
  classical side information, Thm. 2-weak-source-q for quantum);
* ``markov``  -- sources correlated through the adversary's system
  (Cor. MarkovFor2Uni, Thm. Markov1, Thm. Markov2).

Readings where the paper leaves a case implicit:

* quantum side information in the product model for Dodis et al. and
  Trevisan: a product state is a Markov state, so the Markov bound applies
  (the paper gives only the Markov bound for those two);
* classical side information in the Markov model (left out of Fig. Table,
  "computed from Thm. Markov1"): the larger of Thm. Markov1 applied to the
  classical two-source bound (entropies lowered by log2(1/eps0), error
  3 eps0) and the quantum Markov bound, since a quantum-proof extractor is
  also classical-proof;
* a bound below 1 gives m = 0 (nothing can be extracted).
"""

from __future__ import annotations

import math

from .primes import closest_na, is_prime, next_na, prev_na

KINDS = ("toeplitz", "circulant", "dodis", "trevisan")
MODELS = ("seeded", "product", "markov")
ADVERSARIES = ("classical", "quantum")
ADJUST = ("up", "down", "closest")

E = math.e


def _floor0(v: float) -> int:
    return max(0, math.floor(v))


def _largest_m(ok) -> int:
    """Largest integer m >= 1 with ok(m) true, for ok true up to some point and
    false after it; 0 if ok(1) is false.  Bisection over [1, 2^62]."""
    if not ok(1):
        return 0
    lo, hi = 1, 1 << 62
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


def seed_length(kind: str, n1: int, m: int, d: int | None = None) -> int:
    """Seed bits one call takes: n1 + m - 1 (Eq. toep), n1 + 1 (Def. ext-circ),
    n1 (Dodis et al., equal lengths), d (Trevisan)."""
    return {"toeplitz": n1 + m - 1, "circulant": n1 + 1, "dodis": n1, "trevisan": d}[kind]


def trevisan_seed_length(n1: int, m: int, log2_eps: float) -> tuple[int, int, int]:
    """Seed length d = a t^2 of the block weak design (Section "Trevisan"):
    t the smallest prime >= q = 2 ceil(log2 n1 + 2 log2(2m/eps)), and
    a = max(1, ceil((log2(m - 2e) - log2(t - 2e)) / (log2(2e) - log2(2e - 1)))).
    For m <= 2e the logarithm is undefined and a = 1 (reading)."""
    q = 2 * math.ceil(math.log2(n1) + 2 * (1 + math.log2(m) - log2_eps))
    t = q
    while not is_prime(t):
        t += 1
    if m <= 2 * E:
        a = 1
    else:
        num = math.log2(m - 2 * E) - math.log2(t - 2 * E)
        den = math.log2(2 * E) - math.log2(2 * E - 1)
        a = max(1, math.ceil(num / den))
    return t, a, a * t * t


def output_length(kind: str, model: str, adversary: str, n1: int, k1: float,
                  log2_eps: float, k2: float | None = None, d: int | None = None) -> int:
    """Largest output length m the paper's bound allows.

    Toeplitz (Thm. toeplitz and Eq. params:toeplitz-2), Circulant (Thm.
    circSEED and the two-source bound after it), Dodis et al. (the classical
    theorem and the Markov-model theorem of Section "Dodis et al."), Trevisan
    (the combined-parameters theorem and Eq. params:trevisan-2-mm).
    """
    assert kind in KINDS and model in MODELS and adversary in ADVERSARIES
    le = log2_eps
    q = adversary == "quantum"
    L43 = math.log2(4.0 / 3.0)
    if model == "seeded":
        if kind == "toeplitz" or kind == "circulant":
            return _floor0(k1 + 2 * le)
        if kind == "dodis":
            if q:
                return _floor0((k1 + 8 * le + 4 * L43 + 1) / 5)
            return _floor0(k1 + 1 + 2 * le)
        return _largest_m(lambda m: m <= k1 + 4 * le - 4 * math.log2(m) - 6)
    # two-source
    if kind == "circulant":
        n = n1 + 1
        return _floor0(k1 + k2 - n + 2 * le)
    if kind == "toeplitz":
        return _floor0((k1 + k2 - n1 + 1 + 2 * le) / 2)
    if kind == "dodis":
        n = n1
        qm = _floor0((k1 + k2 - n + 8 * le + 4 * L43 + 1) / 5)
        if q:
            return qm
        if model == "product":
            return _floor0(k1 + k2 - n + 1 + 2 * le)
        # Thm. Markov1 with eps0 = eps / 3, entropies k - log2(1/eps0)
        le0 = le - math.log2(3)
        cm = _floor0((k1 + le0) + (k2 + le0) - n + 1 + 2 * le0)
        return max(cm, qm)
    # trevisan
    qm = _largest_m(lambda m: 10 * m <= k1 + 4 * (k2 - d) - 4 * math.log2(m)
                    + 18 * le + 9 * L43 - 6)
    if q:
        return qm
    if model == "product":
        return _largest_m(lambda m: m <= k1 + 4 * k2 - 4 * d + 4 * le - 4 * math.log2(m) - 6)
    le0 = le - math.log2(3)
    cm = _largest_m(lambda m: m <= (k1 + le0) + 4 * ((k2 + le0) - d) + 4 * le0
                    - 4 * math.log2(m) - 6)
    return max(cm, qm)


def plan(kind: str, model: str, adversary: str, n_raw: int, k1: float, log2_eps: float,
         seed_rate: float = 1.0, adjust: str = "up") -> dict:
    """Lengths for extracting from n_raw input bits of min-entropy k1, with a
    seed of min-entropy rate seed_rate (k2 = seed_rate * n2, as in the
    improved QKD and QRNG examples of Section "Cryptomite for ...").

    Circulant needs n1 + 1 in N_A and Dodis et al. n1 in N_A: the input is
    padded with fixed 0 bits up to the next member (Thm. short-seed-ext: fixed
    bits add no entropy, k1 unchanged) or cut down to the previous one
    (Lemma shorten-entropy: k1 drops by the bits cut), per ``adjust``.
    Toeplitz two-source: k2 = r (n1 + m - 1) depends on m; m is the largest
    integer with m <= k1 + (k2 - n2) + 2 log2 eps.  Trevisan: seeded only
    (its two-source seed length depends on m; use output_length with d).
    """
    assert kind in KINDS and adjust in ADJUST
    out = dict(pad_input=0, cut_input=0)
    if kind in ("circulant", "dodis"):
        target = n_raw + 1 if kind == "circulant" else n_raw
        P = {"up": next_na, "down": prev_na, "closest": closest_na}[adjust](target)
        if P >= target:
            out["pad_input"] = P - target
        else:
            out["cut_input"] = target - P
            k1 = max(0.0, k1 - (target - P))
        n1 = P - 1 if kind == "circulant" else P
    else:
        n1 = n_raw
    out["n1"], out["k1"] = n1, k1
    if kind == "trevisan":
        assert model == "seeded"
        m = output_length(kind, model, adversary, n1, k1, log2_eps)
        out["m"] = m
        out["n2"] = trevisan_seed_length(n1, m, log2_eps)[2] if m > 0 else 0
        out["k2"] = float(out["n2"])
        return out
    if kind == "toeplitz":
        if model == "seeded":
            m = output_length(kind, model, adversary, n1, k1, log2_eps)
        else:
            r = seed_rate
            m = _largest_m(lambda m: m <= k1 + (r * (n1 + m - 1) - (n1 + m - 1)) + 2 * log2_eps)
        out["m"] = m
        out["n2"] = n1 + m - 1 if m > 0 else 0
        out["k2"] = out["n2"] * (1.0 if model == "seeded" else seed_rate)
        return out
    n2 = seed_length(kind, n1, 0)
    k2 = float(n2) if model == "seeded" else seed_rate * n2
    out["m"] = output_length(kind, model, adversary, n1, k1, log2_eps, k2=k2)
    out["n2"], out["k2"] = n2, k2
    return out


def vn_expected_length(n: int, p: float) -> float:
    """Expected Von Neumann output length for n IID bits of bias p
    (Section "Von Neumann"): p (1 - p) n."""
    return p * (1 - p) * n
