/*
 * cm_params.h -- output lengths and input/seed lengths of the extractors
 * (host arithmetic, no GPU work), part of libcm.so.
 *
 * The extractors' security statements bound the output length m by the input
 * min-entropy k1, the seed's min-entropy k2 (two-source use) and the error
 * epsilon (Section "Library in detail" of arXiv 2402.09481 and its summary
 * Fig. Table).  These calls evaluate those bounds so that the m passed to
 * cm_toeplitz / cm_circulant / cm_dodis is one the theorems cover, and pick the
 * N_A lengths the Circulant and Dodis et al. constructions require.
 *
 * Conventions: the error is given as log2_eps = log2(epsilon) (< 0), so tiny
 * errors stay representable; entropies are in bits, as doubles; every bound is
 * evaluated in double precision and the floor taken last; a bound below 1
 * yields m = 0 (nothing can be extracted).  n1 is the number of input bits an
 * extraction call takes: the n of cm_toeplitz and cm_dodis, the n of
 * cm_circulant (seed length n1 + 1).  All calls are thread-safe, reentrant and
 * allocate nothing the caller must free.  Errors: CM_EINVAL for a NULL output
 * pointer, an unknown enum value, log2_eps not finite or >= 0, a negative or
 * non-finite entropy, k1 > n1, k2 above the seed length, a Circulant n1 + 1 or
 * Dodis et al. n1 outside N_A, or n1 = 0.
 */
#ifndef CM_PARAMS_H
#define CM_PARAMS_H

#include <stdint.h>

#include "cm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Extractor for the parameter calls: the three of cm_kind, plus Trevisan
 * (Section "Trevisan"), whose lengths are computed here although its
 * extraction is not part of this library. */
#define CM_PARAM_TREVISAN 3

typedef enum {
    CM_MODEL_SEEDED = 0,  /* perfect seed: k2 = n2 */
    CM_MODEL_PRODUCT = 1, /* two independent weak sources (Thm. 2-weak-source, 2-weak-source-q) */
    CM_MODEL_MARKOV = 2   /* sources correlated through the adversary (Cor. MarkovFor2Uni,
                             Thm. Markov1, Thm. Markov2) */
} cm_source_model;

typedef enum { CM_ADV_CLASSICAL = 0, CM_ADV_QUANTUM = 1 } cm_adversary;

/* How cm_plan_params moves a length onto N_A. */
typedef enum {
    CM_ADJUST_UP = 0,     /* next member >= the length: pad the input with 0 bits */
    CM_ADJUST_DOWN = 1,   /* previous member <= the length: cut the input's last bits */
    CM_ADJUST_CLOSEST = 2 /* the nearer of the two; a tie takes the larger */
} cm_adjust;

/*
 * Largest output length m allowed by the paper's bound for `kind`
 * (CM_TOEPLITZ, CM_CIRCULANT, CM_DODIS or CM_PARAM_TREVISAN):
 *
 *   Toeplitz   seeded   m <= k1 + 2 log2 eps                       (Thm. in Sec. "Toeplitz")
 *              two-src  m <= (k1 + k2 - n1 + 1 + 2 log2 eps) / 2   (Eq. params:toeplitz-2)
 *   Circulant  seeded   m <= k1 + 2 log2 eps                       (Thm. circSEED)
 *              two-src  m <= k1 + k2 - (n1 + 1) + 2 log2 eps       (Sec. "Our new Circulant")
 *   Dodis      classical seeded   m <= k1 + 1 + 2 log2 eps         (Sec. "Dodis et al.")
 *              classical product  m <= k1 + k2 - n1 + 1 + 2 log2 eps
 *              quantum (Markov)   m <= (k1 + k2 - n1 + 8 log2 eps + 4 log2(4/3) + 1) / 5,
 *                                 k2 = n1 when seeded
 *   Trevisan   seeded   m <= k1 + 4 log2 eps - 4 log2 m - 6        (Sec. "Trevisan")
 *              classical product  m <= k1 + 4 k2 - 4 d + 4 log2 eps - 4 log2 m - 6
 *              quantum (Markov)   10 m <= k1 + 4 (k2 - d) - 4 log2 m + 18 log2 eps
 *                                         + 9 log2(4/3) - 6     (Eq. params:trevisan-2-mm)
 *
 * Two-source Circulant and Toeplitz take the same bound in both models and for
 * both adversaries (Cor. MarkovFor2Uni).  Quantum side information in the
 * product model takes the Markov bound for Dodis et al. and Trevisan (a
 * product state is a Markov state).  Classical side information in the Markov
 * model takes the larger of Thm. Markov1 applied to the classical two-source
 * bound (entropies lowered by log2(3/eps), error eps/3) and the quantum bound.
 * For Trevisan the implicit bounds are solved for the largest integer m.
 *
 * k2 is ignored when model is CM_MODEL_SEEDED; d (Trevisan seed length, see
 * cm_trevisan_seed_length) is ignored for the other kinds.  *m receives the
 * length (0 if the bound is below 1).
 */
cm_status cm_output_length(int kind, int model, int adversary, uint64_t n1, uint64_t d, double k1,
                           double k2, double log2_eps, int64_t *m);

/*
 * Trevisan seed length of the block weak design (Sec. "Trevisan"): t is the
 * smallest prime >= q = 2 ceil(log2 n1 + 2 log2(2m / eps)),
 * a = max(1, ceil((log2(m - 2e) - log2(t - 2e)) / (log2(2e) - log2(2e - 1))))
 * (a = 1 when m <= 2e, where the logarithm is undefined), d = a t^2.
 * Any of t, a, d may be NULL.  CM_EINVAL if n1 = 0, m = 0 or log2_eps is not
 * finite and negative.
 */
cm_status cm_trevisan_seed_length(uint64_t n1, uint64_t m, double log2_eps, uint64_t *t, uint64_t *a,
                                  uint64_t *d);

/* Result of cm_plan_params. */
typedef struct {
    uint64_t n1;        /* input bits the extraction call takes (its n argument) */
    uint64_t n2;        /* seed bits it takes (Trevisan: d); 0 when m = 0 for Toeplitz */
    uint64_t pad_input; /* fixed 0 bits appended to the raw input (n1 above the raw length) */
    uint64_t cut_input; /* bits removed from the end of the raw input (n1 below it) */
    double k1;          /* input min-entropy after the adjustment */
    double k2;          /* seed min-entropy: seed_rate * n2 (n2 when seeded) */
    int64_t m;          /* output length */
    uint64_t reserved[3];
} cm_param_plan;

/*
 * Lengths for one extraction from n_raw input bits of min-entropy k1, with a
 * seed of min-entropy rate seed_rate in (0, 1] (k2 = seed_rate * n2, as in the
 * paper's improved QKD and QRNG examples; ignored when seeded).
 *
 *   Circulant: n1 + 1 must lie in N_A; Dodis et al.: n1 must.  The target
 *   length (n_raw + 1, resp. n_raw) moves to a member per `adjust`: padding
 *   appends fixed 0 bits and keeps k1 (fixed bits carry no entropy, as in
 *   Thm. short-seed-ext); cutting removes the last bits and lowers k1 by
 *   their number, floored at 0 (Lemma shorten-entropy).
 *   Toeplitz: n1 = n_raw, n2 = n1 + m - 1; in a two-source model k2 depends on
 *   m, and m is the largest integer with m <= k1 + (k2 - n2) + 2 log2 eps.
 *   Trevisan: seeded only (the two-source seed length depends on m; use
 *   cm_output_length with an explicit d); n2 = d for the m found.
 *
 * CM_EINVAL as for cm_output_length, for seed_rate outside (0, 1], for a
 * two-source Trevisan plan, or when no N_A member exists in the direction
 * asked.
 */
cm_status cm_plan_params(int kind, int model, int adversary, uint64_t n_raw, double k1,
                         double seed_rate, double log2_eps, int adjust, cm_param_plan *out);

/* Nearest member of N_A to n: the nearer of cm_prev_na_prime(n) and
 * cm_next_na_prime(n), the larger on a tie; 0 if neither exists. */
uint64_t cm_closest_na_prime(uint64_t n);

#ifdef __cplusplus
}
#endif

#endif /* CM_PARAMS_H */
