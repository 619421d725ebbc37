"""CPU oracle for the Toeplitz, Circulant and Dodis et al. extractors.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library, its Python
binding, the serving loop) imports, links or executes anything in this package.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

The oracle computes the extractors from their matrix definitions in the paper
(Section "Library in detail": Def. ext-circ with Eq. circ-matrix, the Dodis et al.
matrix of Section "Dodis (and Circulant) implementation", Eq. toep-ext and
Eq. toep).  It builds the GF(2) matrix rows explicitly and multiplies them with
the other operand modulo 2.  There is no transform, no field arithmetic and no
code shared with the CUDA path; the two meet only in the seeded input generator
``paper_2402_09481_gb300.inputs``, which holds none of the method's arithmetic.

``oracle.params`` evaluates the output-length theorems of the same Section
(and the Trevisan seed length, the N_A length planning of the paper's QKD and
QRNG examples); ``tests/test_params.py`` pins it to the paper's printed
example arithmetic and re-derives each two-source and Markov-model bound from
its base theorem.

``oracle.von_neumann`` is the Von Neumann extractor of Alg. vn, pinned by
``tests/test_von_neumann_oracle.py``.

``oracle.trevisan`` is the one-bit step of Trevisan's extractor (the
Reed-Solomon-Hadamard one-bit extractor of Section "Trevisan implementation",
with the weak design's sets as an input), pinned by
``tests/test_trevisan_oracle.py``.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(brute force, closed forms, the paper's displayed matrices, the two-universality
count of Thm. 2-univ, the rank lemmas, cross-definition identities) and
``tests/test_primes.py`` (the paper's printed prime pins).  No function is
"parity unpinned".
"""

from .extractors import (  # noqa: F401
    pack_bits,
    unpack_bits,
    toeplitz_matrix,
    circulant_matrix,
    dodis_matrix,
    gf2_matvec,
    toeplitz,
    circulant,
    dodis,
    toeplitz_rows,
    circulant_rows,
    dodis_rows,
    toeplitz_packed,
    circulant_packed,
    dodis_packed,
    DodisPreconditionError,
)
from .primes import (  # noqa: F401
    is_prime,
    has_primitive_root_2,
    ord2_bruteforce,
    next_na,
    prev_na,
    closest_na,
)
