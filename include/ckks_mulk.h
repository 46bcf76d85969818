/*
 * ckks_mulk.h -- C ABI of the GB300 RNS-CKKS multi-input ciphertext
 * multiplication library (libckks_mulk.so).
 *
 * Method: "Multi-Input Ciphertext Multiplication for Homomorphic Encryption"
 * (Akherati and Zhang). The library multiplies k ciphertexts with the
 * paper's k-input multiplier: tensor products of child tuples (Eq. 13),
 * multi-level rescaling at inner nodes (Algorithm 1, Eq. 16-17),
 * relinearisation of d_2..d_n with the extra evaluation keys ek_t
 * (Eq. 14-15) summed before a single ModDown per output polynomial
 * (Section III), the merged INTT and scaled BConv of ModDown (Eq. 11-12),
 * and the relocated rescale at the root (coefficient-domain rs, Eq. 6,
 * followed by one NTT; Section IV).
 *
 * Conventions (all entry points)
 *  - Moduli: q_0..q_{L-1} (Q) and p_0..p_{K-1} (P), every prime < 2^61 and
 *    = 1 mod 2N. "Prime index" x < L means q_x, x >= L means p_{x-L}.
 *  - A polynomial limb is N uint64 residues in [0, q). The NTT domain is the
 *    negacyclic evaluation map A[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q,
 *    psi = the smallest primitive 2N-th root of unity mod q, brv the
 *    log2(N)-bit reversal.
 *  - A tuple (ckks_tuple) is n_polys polynomials of `level` limbs each,
 *    limb-major: limb j of polynomial a starts at
 *    data + (a * poly_stride + j) * N. A ciphertext has n_polys = 2.
 *  - Device pointers are caller-owned device memory on the context's device;
 *    the library never frees them. Calls are asynchronous and ordered on the
 *    given CUDA stream (a cudaStream_t passed as void*; NULL = default
 *    stream). Inputs must stay valid until the stream reaches the call.
 *  - Evaluation keys for t = 2..t_max, digit beta < dnum:
 *    keys[t-2][beta][l][x][N] (l = 0, 1; x = prime index, Q rows first),
 *    NTT domain, with ek_{t,beta} = (-a s + e + [x < L] P G_beta s^t, a),
 *    G_beta = Qhat_beta [Qhat_beta^-1]_{Q_beta}, Qhat_beta = Q / Q_beta,
 *    digit beta = primes q_{beta alpha} .. q_{(beta+1) alpha - 1},
 *    alpha = ceil(L / dnum). For dnum = 1 this is Eq. 2, 9 and 14.
 *  - Errors: every entry point returns 0 (CKKS_OK) or a negative code;
 *    nothing throws across the ABI. A CUDA launch error is returned as
 *    CKKS_ECUDA and also kept as a sticky status (ckks_check).
 *  - Workspace: the caller allocates it (ckks_workspace_size); the library
 *    allocates no device memory after context creation.
 */
#ifndef CKKS_MULK_H
#define CKKS_MULK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CKKS_OK 0
#define CKKS_EINVAL (-1)   /* bad argument: shape, level, flag, partition */
#define CKKS_ELEVEL (-2)   /* level too low for the partition depth, or > L */
#define CKKS_EKEY (-3)     /* evaluation-key set lacks ek_t for a needed t */
#define CKKS_ENOMEM (-4)   /* workspace smaller than ckks_workspace_size */
#define CKKS_ECUDA (-5)    /* CUDA error (launch or sticky) */
#define CKKS_ETIMEOUT (-6) /* a bounded device wait ran out */
#define CKKS_EBUSY (-7)    /* admission refused */
#define CKKS_ECHECK (-8)   /* integrity check failed: a residue >= q, or resident keys changed */

typedef struct ckks_context ckks_context;
typedef struct ckks_evk_set ckks_evk_set;
typedef struct ckks_plan ckks_plan;

typedef struct {
    uint32_t log_n;     /* N = 2^log_n, 4 <= log_n <= 16 */
    uint32_t L;         /* number of Q primes, 1 <= L, L + K <= 64 */
    uint32_t K;         /* number of P primes */
    uint32_t dnum;      /* key-switching digits, 1 <= dnum <= L */
    const uint64_t *q;  /* host array [L] */
    const uint64_t *p;  /* host array [K] */
} ckks_params;

typedef struct {
    uint64_t *data;       /* device, see "tuple" above */
    uint32_t n_polys;     /* 2 for a ciphertext, n + 1 for a product of n */
    uint32_t level;       /* active limbs q_0..q_{level-1} */
    uint32_t poly_stride; /* limbs between polynomials, >= level */
    uint32_t ntt_form;    /* 1 = NTT domain (required by ckks_mul_k) */
    double scale;         /* tracked on the host; not used by the kernels */
} ckks_tuple;

typedef struct {
    uint64_t limb_ntt;     /* limb forward transforms enqueued */
    uint64_t limb_intt;    /* limb inverse transforms enqueued */
    uint64_t ntt_phase;    /* forward transform kernel launches */
    uint64_t intt_phase;   /* inverse transform kernel launches */
    uint64_t bconv;        /* basis conversions (ModUp digits and ModDowns) */
    uint64_t kernels;      /* every kernel launch */
} ckks_op_counters;

/* ---------------------------------------------------------------- context
 * ckks_context_create: validates the parameters (primes < 2^61, prime,
 * = 1 mod 2N, pairwise distinct) and builds the twiddle, BConv, rescale
 * (Eq. 16) and key-preparation tables on `device`. The context owns these
 * tables (one device allocation) until ckks_context_destroy.
 * Returns CKKS_EINVAL for bad parameters, CKKS_ECUDA if the device
 * allocation fails. */
int ckks_context_create(const ckks_params *params, int device, ckks_context **out);
void ckks_context_destroy(ckks_context *ctx);

/* ---------------------------------------------------------------- keys
 * ckks_keygen_evk: evaluation keys for t = 2..t_max from the secret s
 * (device int64 [N], coefficients in {-1, 0, 1}), the masks a (device
 * [t_max-1][dnum][L+K][N] residues, NTT domain) and the errors e (device
 * int64 [t_max-1][dnum][N]); writes keys [t_max-1][dnum][2][L+K][N] in the
 * layout of the conventions (Eq. 2, 9, 14 with the digit gadget).
 * Workspace: ckks_keygen_workspace_size bytes. */
int ckks_keygen_workspace_size(const ckks_context *ctx, size_t *bytes);
int ckks_keygen_evk(ckks_context *ctx, uint32_t t_max, const int64_t *s, const uint64_t *a, const int64_t *e,
                    uint64_t *keys, void *workspace, size_t ws_bytes, void *stream);

/* ckks_evk_set_create: adopts a key buffer in the layout above for
 * t = 2..t_max; the buffer must be 16-byte aligned (CKKS_EINVAL otherwise:
 * the key MAC reads it with 16-byte loads). The buffer is converted IN
 * PLACE to the library's internal form (Montgomery form; P^-1 folded into
 * the Q rows, Eq. 12) and is borrowed until ckks_evk_set_destroy; do not
 * read it as plain keys after. */
int ckks_evk_set_create(ckks_context *ctx, uint32_t t_max, uint64_t *keys, void *stream, ckks_evk_set **out);
void ckks_evk_set_destroy(ckks_evk_set *set);

/* Integrity checks (failure detection; the paper has no counterpart).
 * ckks_evk_set_create also takes a position-dependent 64-bit checksum of
 * the prepared keys (it synchronises `stream` once for that);
 * ckks_evk_verify recomputes it and returns CKKS_ECHECK if the resident
 * keys changed since (a stray write into the borrowed buffer), CKKS_OK if
 * not. Synchronous on `stream`. */
int ckks_evk_verify(ckks_evk_set *set, void *stream);

/* ------------------------------------------------------ around the product
 * Section II's public key, encryption and decryption, on the device.
 * ckks_public_key: pk = (-a s + e, a) on the L Q limbs, NTT domain; s, e
 * device int64 [N] (small), a device [L][N] residues (NTT domain), pk device
 * [2][L][N]. ckks_encrypt: out = (v pk_0 + e_0 + m, v pk_1 + e_1) on limbs
 * 0..level-1, NTT domain; m, v, e_0, e_1 device int64 [N] (|m| < 2^62: the
 * integer message polynomial, e.g. scaled and rounded canonical-embedding
 * coefficients). ckks_decrypt: c_0 + c_1 s on the lowest two limbs (one at
 * level 1), lifted by CRT to [0, q_0 q_1) and centred, written as double
 * [N] (device); exact while |message| < q_0 q_1 / 2. Workspace for all
 * three: ckks_encrypt_workspace_size. */
int ckks_encrypt_workspace_size(const ckks_context *ctx, size_t *bytes);
/* Canonical-embedding encoding and decoding (Section II), N/2 complex slots
 * per message, slot j at zeta_j = exp(i pi 5^j / N). ckks_encode: z device
 * double [batch][N/2][2] (re, im) -> m device int64 [batch][N], m_i =
 * round((2/N) Re sum_j scale z_j zeta_j^-i) (round half to even), computed
 * in double precision by a four-step FFT, so m carries the FFT's rounding
 * (about log2(N) ulps of scale |z|); |scale z| must stay below 2^62.
 * ckks_decode: m device double [batch][N] (e.g. ckks_decrypt's output)
 * -> z device double [batch][N/2][2], z_j = sum_i m_i zeta_j^i / scale.
 * Workspace (16-byte aligned): ckks_embed_workspace_size(batch) bytes.
 * CKKS_EINVAL for batch 0 or above 65535, scale <= 0, N < 4. Both are
 * asynchronous on `stream`. */
int ckks_embed_workspace_size(const ckks_context *ctx, uint32_t batch, size_t *bytes);
int ckks_encode(ckks_context *ctx, const double *z, uint32_t batch, double scale, int64_t *m, void *workspace,
                size_t ws_bytes, void *stream);
int ckks_decode(ckks_context *ctx, const double *m, uint32_t batch, double scale, double *z, void *workspace,
                size_t ws_bytes, void *stream);
int ckks_public_key(ckks_context *ctx, const int64_t *s, const uint64_t *a, const int64_t *e, uint64_t *pk,
                    void *workspace, size_t ws_bytes, void *stream);
int ckks_encrypt(ckks_context *ctx, const int64_t *m, const int64_t *v, const int64_t *e0, const int64_t *e1,
                 const uint64_t *pk, uint32_t level, ckks_tuple *out, void *workspace, size_t ws_bytes,
                 void *stream);
int ckks_decrypt(ckks_context *ctx, const ckks_tuple *ct, const int64_t *s, double *out, void *workspace,
                 size_t ws_bytes, void *stream);
/* Batched forms, one set of launches for many messages (the single calls
 * above are batch 1). ckks_encrypt_batch: m, v, e_0, e_1 device int64
 * [batch][N]; out[batch] evenly spaced tuples (one poly stride) at `level`.
 * Workspace: ckks_encrypt_batch_workspace_size(level, batch) bytes (the
 * messages are processed in chunks of up to 65535 / (4 level)).
 * ckks_decrypt_batch: ct[batch] evenly spaced, same level and poly stride;
 * out device double [batch][N]; batch <= 32767. Workspace:
 * ckks_decrypt_batch_workspace_size(batch). Errors as for the single calls. */
int ckks_encrypt_batch_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes);
int ckks_encrypt_batch(ckks_context *ctx, const int64_t *m, const int64_t *v, const int64_t *e0, const int64_t *e1,
                       uint32_t batch, const uint64_t *pk, uint32_t level, ckks_tuple *out, void *workspace,
                       size_t ws_bytes, void *stream);
int ckks_decrypt_batch_workspace_size(const ckks_context *ctx, uint32_t batch, size_t *bytes);
int ckks_decrypt_batch(ckks_context *ctx, const ckks_tuple *ct, uint32_t batch, const int64_t *s, double *out,
                       void *workspace, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------- rotation
 * Slot rotation by a Galois automorphism sigma_g: a(X) -> a(X^g), g odd,
 * 1 <= g < 2N (Section II's canonical embedding: g = 5^r mod 2N moves slot
 * j + r to slot j, g = 2N - 1 conjugates every slot). Key switching back to
 * s reuses the relinearisation steps (ModUp, key MAC, ModDown) with one key.
 * ckks_galois_element: g = 5^r mod 2N for any integer r (r < 0 rotates
 * the other way). CKKS_EINVAL for N < 4.
 * ckks_automorphism: out = sigma_g(in) for every polynomial of an NTT-domain
 * tuple (a permutation of each limb: out[i] = in[brv((g (2 brv(i) + 1) mod
 * 2N - 1) / 2)]); same level and scale; out must not overlap in
 * (CKKS_EINVAL if out->data == in->data; partial overlap is undefined).
 * ckks_keygen_galois: the Galois key of g from s, a, e (layouts as in
 * ckks_keygen_evk with t_max = 2: a device [dnum][L+K][N], e device int64
 * [dnum][N], keys [dnum][2][L+K][N]): gk_beta = (-a_beta s + e_beta +
 * [Q limb] P G_beta sigma_g(s), a_beta). Workspace:
 * ckks_keygen_workspace_size. Adopt it with ckks_evk_set_create(ctx, 2,
 * keys, ...): a Galois key is a one-key set whose key sits where ek_2 would.
 * ckks_rotate / ckks_rotate_batch: out = (sigma c_0 + [P^-1 sigma(c_1)
 * gk_0], [P^-1 sigma(c_1) gk_1]) with ModDown finished in the NTT domain;
 * same level and scale as the input; decrypts under s to sigma_g of the
 * message. Batch tuples evenly spaced as in ckks_mul2_batch; out may be
 * the input. Workspace: ckks_rotate_workspace_size. Errors: CKKS_EINVAL
 * (g even or >= 2N, shapes), CKKS_ELEVEL, CKKS_ENOMEM. */
int ckks_galois_element(const ckks_context *ctx, int32_t r, uint32_t *g);
int ckks_automorphism(ckks_context *ctx, const ckks_tuple *in, uint32_t g, ckks_tuple *out, void *stream);
int ckks_keygen_galois(ckks_context *ctx, uint32_t g, const int64_t *s, const uint64_t *a, const int64_t *e,
                       uint64_t *keys, void *workspace, size_t ws_bytes, void *stream);
int ckks_rotate_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes);
int ckks_rotate(ckks_context *ctx, const ckks_tuple *in, uint32_t g, const ckks_evk_set *gk, ckks_tuple *out,
                void *workspace, size_t ws_bytes, void *stream);
int ckks_rotate_batch(ckks_context *ctx, const ckks_tuple *in, uint32_t batch, uint32_t g, const ckks_evk_set *gk,
                      ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- plans
 * ckks_plan_create: the partition tree of a k-input multiply (2 <= k <= 12)
 * in the notation of Table II, e.g. "(4,3)|(2,2)": '|' separates layers and
 * each group list of a layer splits, left to right, the next group of the
 * layer above with the same size. NULL selects Table II's optimised
 * partition. CKKS_EINVAL if the text does not parse or breaks the depth rule
 * (Section V-C: rescales on any path <= ceil(log2 k)). */
int ckks_plan_create(ckks_context *ctx, uint32_t k, const char *partition, ckks_plan **out);
void ckks_plan_destroy(ckks_plan *plan);
/* depth = rescales on the longest path (output level = input level - depth);
 * rs_units = Table II's rescale-unit count below the root. */
int ckks_plan_describe(const ckks_plan *plan, uint32_t *depth, uint32_t *rs_units, uint32_t *n_nodes);

/* Partition search (Section V-C: among the partitions that keep the depth at
 * ceil(log2 k), find the one of lowest complexity). Every valid tree for
 * k inputs (2 <= k <= 12) is enumerated and costed by `criterion`:
 * 0 = Table II's rescale-unit count; 1 = limb (I)NTTs of the whole k-input
 * multiply at input `level` with K special primes and digits of `alpha`
 * primes (Algorithm 1 at inner nodes, relinearisation and relocated rescale
 * at the root); 2 = precision: 10^6 x the largest degree of a tuple that an
 * inner node rescales before relinearisation, plus criterion 1's count (the
 * rounding error of a rescaled degree-t tuple decrypts multiplied by s^t,
 * so the decoded product loses about log2 |s| bits per degree; not a
 * criterion of the paper). The cheapest tree's text (layered notation, NUL-terminated)
 * is written to `text` (text_len bytes) and its cost to *cost; ties go to
 * fewer nodes, then the smaller text. The text is parsed back before it is
 * returned, so ckks_plan_create accepts it. ckks_plan_cost gives the same
 * cost for an existing plan. Host only: no device work. */
int ckks_plan_optimize(uint32_t k, int criterion, uint32_t level, uint32_t K, uint32_t alpha, char *text,
                       size_t text_len, double *cost);
int ckks_plan_cost(const ckks_plan *plan, int criterion, uint32_t level, uint32_t K, uint32_t alpha, double *cost);

/* Workspace bytes for ckks_mul_k / ckks_mul_k_batch at this input level and
 * batch size. CKKS_ELEVEL if level <= depth or level > L. */
int ckks_workspace_size(const ckks_context *ctx, const ckks_plan *plan, uint32_t level, uint32_t batch,
                        size_t *bytes);

/* ---------------------------------------------------------------- multiply
 * ckks_mul_k: out = product of the k ciphertexts ct[0..k-1] (all NTT domain,
 * same level) with the plan's tree. out->data must hold 2 polynomials of
 * level - depth limbs (poly_stride >= that); out is written in the NTT
 * domain and out->level / out->scale are set (scale = product of input
 * scales / product of the divided primes). The result equals, residue for
 * residue, the oracle's evaluation: inner nodes rescaled mu = m-1 times,
 * root relinearised with ek_2..ek_n then rescaled m-1 times.
 * CKKS_EKEY if the set's t_max < k. */
int ckks_mul_k(ckks_context *ctx, const ckks_tuple *ct, uint32_t k, const ckks_evk_set *evk,
               const ckks_plan *plan, ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream);

/* ckks_mul_k_batch: `batch` independent products with one plan and one key
 * set, each kernel launch covering the whole batch. ct is [batch][k] tuples,
 * out is [batch]. For every input position u, ct[b*k+u].data must be
 * ct[u].data + b * stride_u for one stride_u (likewise for out, whose
 * stride must not be 0: two batch elements cannot share one output, which
 * is CKKS_EINVAL; inputs may repeat); the same level, poly_stride and
 * n_polys for all b. The batched calls below follow the same rule. */
int ckks_mul_k_batch(ckks_context *ctx, const ckks_tuple *ct, uint32_t k, uint32_t batch, const ckks_evk_set *evk,
                     const ckks_plan *plan, ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream);

/* Uneven work in one call (Section V: products of different k, partitions
 * and levels): each request is one ckks_mul_k_batch group (same k, plan and
 * level inside it, its own batch stride). ckks_mul_k_requests enqueues the
 * groups in order on `stream`, reusing one workspace of
 * ckks_requests_workspace_size bytes (the largest group's need); it
 * allocates nothing and does not synchronise (unless the "check_residues"
 * tunable is on). On an error it returns that group's code and *done (if
 * not NULL) gives the number of groups enqueued before it. The Python
 * executor builds such groups from arbitrary requests and replays them from
 * a CUDA graph over several streams. */
typedef struct {
    const ckks_tuple *ct;       /* [batch][k] input tuples */
    uint32_t k, batch;
    const ckks_evk_set *evk;
    const ckks_plan *plan;      /* partition tree for k inputs */
    ckks_tuple *out;            /* [batch] outputs */
} ckks_request;
int ckks_requests_workspace_size(const ckks_context *ctx, const ckks_request *req, uint32_t n, size_t *bytes);
int ckks_mul_k_requests(ckks_context *ctx, const ckks_request *req, uint32_t n, uint32_t *done, void *workspace,
                        size_t ws_bytes, void *stream);

/* Cross-shape batches ("waves", Section V's k-input products in any mix of
 * k, partition and level, as one set of launches). A wave holds n products
 * of one context: item i multiplies ct[0..k-1] (2 polynomials each, NTT
 * form, one level) along `plan` into `out` (2 polynomials, level - depth),
 * with the same residues as ckks_mul_k on that item alone. Inner tree nodes
 * of all products are grouped by height and every stage (tensor product,
 * Algorithm 1's transforms and rescale chain; at the roots ModUp, BConv,
 * the key MAC of Eq. 15, ModDown of Eq. 11 / 12 and the relocated rescale)
 * is one launch over every product with work there, its entries read from
 * device tables. The paper's forms are always used (the "inner_rescale",
 * "root_rescale", "moddown" and "check_residues" tunables do not apply).
 *
 * ckks_wave_create validates the items (as ckks_mul_k) and keeps their
 * pointers (the wave borrows them: inputs and outputs must stay allocated
 * while it is used); CKKS_EINVAL also for N <= 256 and for two items sharing
 * one output. ckks_wave_workspace_size gives the bytes of the two device
 * buffers a run needs: the job tables and the products' scratch. Waves run
 * one after another on one stream may share a scratch buffer; each keeps
 * its own table buffer. ckks_wave_run enqueues the wave on `stream` (both
 * buffers 256-byte aligned); the first run with a given pair of buffers
 * writes the job tables with one host-to-device copy on the stream (later
 * runs with the same pair reuse them), so that first run should not be
 * inside a stream capture. ckks_wave_describe returns the number of
 * launches of a run and the number of inner-node heights (valid after the
 * first run). ckks_wave_destroy waits for the wave's table copy, if one is
 * in flight, and frees its host staging buffer. No device memory is
 * allocated by the library. */
typedef struct ckks_wave ckks_wave;
typedef struct {
    const ckks_tuple *ct;       /* k input ciphertexts */
    uint32_t k;
    const ckks_plan *plan;      /* partition tree for k inputs */
    ckks_tuple *out;            /* output; level, scale and form are set by ckks_wave_run */
} ckks_wave_item;
int ckks_wave_create(ckks_context *ctx, const ckks_wave_item *items, uint32_t n, const ckks_evk_set *evk,
                     ckks_wave **out);
int ckks_wave_workspace_size(const ckks_wave *w, size_t *table_bytes, size_t *scratch_bytes);
int ckks_wave_run(ckks_wave *w, void *tables, size_t table_bytes, void *scratch, size_t scratch_bytes, void *stream);
int ckks_wave_describe(const ckks_wave *w, uint32_t *n_launches, uint32_t *heights);
void ckks_wave_destroy(ckks_wave *w);

/* ckks_mul2: the standard 2-input multiply of Section II (Eq. 1-7): tensor
 * product, relinearisation with ModDown finished in the NTT domain, one RS in
 * the NTT domain (Eq. 7). The comparator for chained multiplication. Output
 * level = min input level - 1. Workspace: ckks_mul2_workspace_size.
 * ckks_mul2_batch: `batch` such products; a, b and out are [batch] arrays
 * with a constant pointer stride each (as in ckks_mul_k_batch). */
int ckks_mul2_workspace_size(const ckks_context *ctx, uint32_t level, uint32_t batch, size_t *bytes);
int ckks_mul2(ckks_context *ctx, const ckks_tuple *a, const ckks_tuple *b, const ckks_evk_set *evk,
              ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream);
int ckks_mul2_batch(ckks_context *ctx, const ckks_tuple *a, const ckks_tuple *b, uint32_t batch,
                    const ckks_evk_set *evk, ckks_tuple *out, void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- steps
 * ckks_tensor (Eq. 13): out = product of m tuples (NTT domain, coefficient-
 * wise in each limb), out->n_polys = sum(n_polys) - m + 1, level = min
 * input level (higher inputs drop their top limbs). */
int ckks_tensor(ckks_context *ctx, const ckks_tuple *in, uint32_t m, ckks_tuple *out, void *stream);

/* ckks_relin (Eq. 15 with the combined ModDown): d has n + 1 polynomials
 * (NTT domain, n >= 2, ek_t for t <= n needed); out (2 polynomials, same
 * level) gets (d_0, d_1) + sum_t ceil(P^-1 d_t ek_t), in the coefficient
 * domain if out_ntt = 0 (Eq. 11 merged form), else NTT domain.
 * Workspace: ckks_relin_workspace_size. */
int ckks_relin_workspace_size(const ckks_context *ctx, uint32_t n, uint32_t level, size_t *bytes);
int ckks_relin(ckks_context *ctx, const ckks_tuple *d, const ckks_evk_set *evk, uint32_t out_ntt, ckks_tuple *out,
               void *workspace, size_t ws_bytes, void *stream);

/* ckks_rescale_multi (Algorithm 1): mu combined rescales of every polynomial
 * of `in` (NTT domain) -> out (level - mu, NTT domain); mu = 1 is Eq. 7.
 * in and out may be the same tuple. Workspace:
 * ckks_rescale_workspace_size. */
int ckks_rescale_workspace_size(const ckks_context *ctx, uint32_t n_polys, uint32_t level, uint32_t mu,
                                size_t *bytes);
int ckks_rescale_multi(ckks_context *ctx, const ckks_tuple *in, uint32_t mu, ckks_tuple *out, void *workspace,
                       size_t ws_bytes, void *stream);
/* ckks_rescale (Eq. 7): one rescale of every polynomial, NTT domain in and
 * out (level - 1); ckks_rescale_multi with mu = 1, same workspace rule. */
int ckks_rescale(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *workspace, size_t ws_bytes,
                 void *stream);

/* ckks_rescale_multi_noalloc: the result of ckks_rescale_multi (Algorithm 1,
 * always that form, whatever the context's "inner_rescale" setting), for
 * callers that cannot allocate device memory where they need a rescale: a
 * component that only receives device pointers from another one and has no
 * allocator of its own, or a loop that must not call cudaMalloc (which can
 * synchronise the device) or take a caching allocator's locks. The paper has
 * no counterpart: this is an interface for such callers. Its scratch is a
 * fixed device array inside the library, ckks_rescale_noalloc_capacity()
 * bytes (32 MiB: a 2-polynomial tuple at N = 2^16 and level 32 fits
 * exactly), held on every device that loads the library until exit; the call
 * makes no cudaMalloc / cudaFree or other allocation. Inputs and outputs are
 * still the caller's (in and out may be the same tuple). The first call on a
 * device resolves the array's device address (once per device, with that
 * device current); make that first call before any stream capture. The
 * caller's current device is the same after the call as before it. Sizes
 * whose scratch exceeds the capacity are rejected with CKKS_ENOMEM. All calls
 * share the one array: calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and must be ordered by the
 * caller. While the context's timing hook is on the call returns
 * CKKS_EINVAL. */
size_t ckks_rescale_noalloc_capacity(void);

int ckks_rescale_multi_noalloc(ckks_context *ctx, const ckks_tuple *in, uint32_t mu, ckks_tuple *out, void *stream);

/* Forward / inverse transform of every limb of a tuple (in and out may be
 * the same tuple); sets out->ntt_form. */
int ckks_ntt(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *stream);
int ckks_intt(ckks_context *ctx, const ckks_tuple *in, ckks_tuple *out, void *stream);

/* ---------------------------------------------------------------- status
 * ckks_counters: operation counts enqueued since the last reset (reset != 0
 * clears them after reading). Counts are taken on the host when work is
 * enqueued, so they need no GPU to read. */
int ckks_counters(ckks_context *ctx, ckks_op_counters *out, int reset);
/* Kernel timing hook (tracing). ckks_profile_enable(ctx, 1) clears earlier
 * records and, until ckks_profile_enable(ctx, 0), records a CUDA event pair
 * on the launch stream around every kernel the library enqueues (events
 * are created by the library on first use, never device memory).
 * ckks_profile_read waits for the recorded events and returns, per kernel
 * class, the launch count, the summed event time, the summed algorithmic
 * bytes (each input and output limb of a launch counted once) and the summed
 * integer work: for the NTT / INTT phases the 64-bit Shoup products (one per
 * butterfly, log2(n)/2 per element of an n-point phase, plus one per element
 * for each fused scaling), for BConv and the key MAC the 64 x 64 -> 128-bit
 * multiply-accumulates (Eq. 4 and Eq. 15 summed term by term), for the
 * tensor product (Eq. 13) its 64 x 64 products and modular reductions; 0
 * for the other classes. */
typedef struct {
    char name[24];
    uint64_t launches;
    double total_ms;
    double alg_bytes;
    double int_ops;
} ckks_kernel_stats;
int ckks_profile_enable(ckks_context *ctx, int enable);
int ckks_profile_read(ckks_context *ctx, ckks_kernel_stats *out, uint32_t max, uint32_t *n_out);

/* Host-to-device transfer by the GPU's own loads (no counterpart in the
 * paper; used to move a step's inputs when that beats the copy engines).
 * ckks_host_device_pointer returns the device address of pinned host
 * memory (CKKS_EINVAL if `host` is not pinned and mapped).
 * ckks_pull copies `bytes` (a multiple of 16; both addresses 16-byte
 * aligned) from src to dst with a grid of `blocks` CTAs of 64 threads on
 * `stream`; either
 * address may be device memory or mapped pinned host memory. Caller-owned
 * buffers; asynchronous. */
int ckks_host_device_pointer(void *host, void **dev);
int ckks_pull(void *dst, const void *src, size_t bytes, int blocks, void *stream);

/* Integer-arithmetic peaks (measurement support; no counterpart in the
 * paper). ckks_peak_int launches blocks x threads threads (threads a
 * multiple of 32, at most 256) that each run ckks_peak_chains() independent
 * chains of `iters` operations of one kind on registers only, and write one
 * word per thread to `out` (device, blocks x threads words, caller-owned):
 *   kind 0  lazy Shoup product x w - floor(x w' / 2^64) q (w' = floor(w 2^64 / q))
 *   kind 1  lazy Cooley-Tukey butterfly of the NTT (Shoup product plus
 *           Harvey's additions and correction)
 *   kind 2  64 x 64 -> 128-bit multiply-accumulate
 *   kind 3  Montgomery product, R = 2^64
 *   kind 4  16 x 16 transpose of 64-bit values within each half-warp by
 *           warp shuffles (the exchange between two radix-16 NTT passes)
 *   kind 5  the same transpose through shared memory
 *   kind 6  kind 1 with the Shoup product's form for q = 1 (mod 2^32)
 *   kind 7  kind 0 in that form
 * (kinds 6 and 7 need q = 1 (mod 2^32), else CKKS_EINVAL before any launch;
 * kinds 4 and 5 run 16 values per thread and count one operation per
 * value moved: blocks x threads x 16 x iters; q, w, wp are not used)
 * q: odd modulus below 2^62; w, wp: host arrays of ckks_peak_chains() Shoup
 * pairs (w < q). The caller times the launch on `stream` with CUDA events:
 * operations per second = blocks x threads x chains x iters / time
 * (kinds 0-3, 6, 7).
 * Returns CKKS_EINVAL for bad arguments, CKKS_ECUDA on a launch error. */
int ckks_peak_chains(void);
int ckks_peak_int(int kind, uint64_t q, const uint64_t *w, const uint64_t *wp, int blocks, int threads, int iters,
                  uint64_t *out, void *stream);

/* Launch tunables of a context; results are the same for every value.
 * Chosen by the autotuner: "ntt_tile_cols" / "ntt_tile_blocks" = elements
 * per CTA tile of the NTT's column / block phases ("ntt_tile" sets both;
 * reading it gives the column value) (1024..8192,
 * power of two; default 4096), "bconv_threads" = threads per BConv block
 * (64..1024, multiple of 32; default 256), "mac_threads" = threads per
 * key-MAC block (same range).
 * Forms of the rescaling, for measuring the paper's reformulations (every
 * rescaling form gives the same residues): "inner_rescale" 0 = Algorithm 1 (mu INTT
 * + (l - mu) NTT per polynomial, default), 1 = mu single rescales of Eq. 7,
 * 2 = INTT of every limb, mu rescales of Eq. 6, NTT of the survivors (Table
 * IV's baseline: l INTT + (l - mu) NTT); "root_rescale" 0 = relocated
 * (Section IV: merged ModDown INTT, coefficient-domain rs, one NTT;
 * default), 1 = prior (ModDown finished in the NTT domain, then the root's
 * rescales by Eq. 7). Form of the key switching (Section III): "moddown"
 * 0 = the key products of every ek_t summed before one ModDown (Eq. 15,
 * default), 1 = one ModDown per ek_t, the results summed (the form Eq. 15
 * replaces; its residues differ from the combined form's by the same small
 * integer W in [0, K (n - 2)] in every limb, the extra wraps of Eq. 5's
 * P-residues; it needs no more workspace). CKKS_EINVAL for an unknown key
 * or a value out of range.
 * Debugging aids: "check_residues" 1 = ckks_mul_k / ckks_mul_k_batch count
 * residues outside [0, q) in their inputs and after every stage (tensor
 * product, Algorithm 1 rescale, relinearisation, root rescale), then
 * synchronise the stream and return CKKS_ECHECK if any were found (results
 * are still written). The count lives in one word per context: checking
 * calls (and ckks_check_residues, ckks_evk_verify) that run at the same
 * time on one context, on different streams, share it and may report each
 * other's violations. "nvtx" 1 = NVTX ranges around each stage's launches,
 * for profilers that filter by range. Both default to 0.
 * Form of the modular products: when every prime of the context (Q and P)
 * is 1 (mod 2^32), "q1_forms" 1 (default) lets the kernels compute the
 * Shoup quotient product and Montgomery's q^-1 and quotient products with
 * 32-bit multiplies (q = h 2^32 + 1); 0 keeps the general 64-bit forms.
 * Residues are the same either way; for other primes the value has no
 * effect.
 * Tensor product kernels (Eq. 13): "tensor_fixed" 1 (default) runs the
 * product of a tree node whose two or three children are all tuples of at
 * least four terms, in one of the compiled shapes (two children of 4..7
 * terms; three of 4 or 5), through a kernel unrolled for exactly that
 * shape; 0 sends every node to the kernels bounded by the largest tuple
 * size. Residues are the same either way. */
int ckks_tune_set(ckks_context *ctx, const char *key, int value);
int ckks_tune_get(const ckks_context *ctx, const char *key, int *value);

/* ckks_check: CKKS_ECUDA if a CUDA error is pending on the context's device
 * (sticky launch error or cudaGetLastError), else CKKS_OK. */
int ckks_check(ckks_context *ctx);
/* ckks_check_residues: *bad = number of residues outside [0, q_j) in the
 * tuple's active limbs (limb j checked against q_j). Synchronous on
 * `stream`; a valid tuple gives 0. */
int ckks_check_residues(ckks_context *ctx, const ckks_tuple *t, uint64_t *bad, void *stream);
const char *ckks_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CKKS_MULK_H */
