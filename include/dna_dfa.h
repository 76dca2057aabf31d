/*
 * dna_dfa.h -- C ABI of the GB300 DNA automaton scan library (libdnadfa.so).
 *
 * The library runs a deterministic finite automaton over a DNA byte sequence on one
 * GPU, following Memeti & Pllana, "Analyzing large-scale DNA Sequences on Multi-core
 * Architectures" (CSE 2015):
 *   - the automaton is the quintuple (Q, Sigma, delta, q0, F) of Sec. II, over the
 *     alphabet A, C, G, T, with q0 = state 0;
 *   - the input is split into chunks (input-based partitioning, Sec. III-A, Fig. 1a);
 *     each chunk's unknown start state is speculated from the symbols before it
 *     (the possible-starting-state idea of Sec. III-A), every chunk is scanned in
 *     parallel, and a join links each chunk's last state to the next chunk's first
 *     state (the "binary reduction" of Sec. III-A); a wrong speculation is repaired
 *     at the converging point (Sec. III-B.3, Alg. 1), where a run from the true state
 *     meets the speculative run after the same number of symbols;
 *   - the result is the exact count of match end positions and, optionally, the
 *     positions themselves (Sec. III-A: counting and extracting k-mers).
 *
 * Semantics every entry point shares (the definition the results must equal):
 *   Each byte is one symbol. A/a, C/c, G/g, T/t are the four bases; any other byte
 *   (N, IUPAC codes, newline, ...) is a reset symbol that sends every state to state
 *   0. The scan starts in state 0, takes one transition per byte and tests the
 *   post-transition state against F (Alg. 1 tests the state after each transition).
 *   The count is the number of such steps that land in F; the positions are the
 *   0-based byte indices of those steps, strictly ascending. For a compiled pattern
 *   this reports every j such that some non-empty substring ending at j, with no
 *   reset byte inside, is a word of the pattern (overlapping occurrences included,
 *   Sec. II).
 *
 * Threading and ownership: handles may be used from several host threads at once;
 * calls on different streams may overlap. The caller owns every sequence and output
 * buffer. Device results are written asynchronously on the given stream and are
 * valid once the stream has completed the call's work.
 *
 * Errors: every entry point returns DNA_OK (0) or a negative DNA_ERR_* code.
 * Argument errors are detected before any work is queued and leave outputs untouched.
 */
#ifndef DNA_DFA_H
#define DNA_DFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers. 0 = the legacy default stream. */
typedef struct CUstream_st *dna_stream_t;

#define DNA_OK                 0
#define DNA_ERR_INVALID_ARG   -1  /* null pointer, n_states = 0, entry >= n_states, bad size */
#define DNA_ERR_NOMEM         -2  /* a host or device allocation failed */
#define DNA_ERR_CAPACITY      -3  /* a fixed capacity (states, batch shape) was exceeded */
#define DNA_ERR_TIMEOUT       -4  /* a bounded device wait gave up (status word) */
#define DNA_ERR_CUDA          -5  /* a CUDA runtime call failed */
#define DNA_ERR_SYNTAX        -6  /* pattern syntax error (host compiler) */
#define DNA_ERR_EMPTY_WORD    -7  /* pattern language contains the empty word */
#define DNA_ERR_NO_DEVICE     -8  /* no usable CUDA device / wrong architecture */

typedef struct dna_dfa dna_dfa; /* opaque; its tables live in device memory */

/*
 * dfa_load -- copies a complete DFA to the current CUDA device (Sec. II quintuple).
 *   table       host, row-major uint32 [n_states][4], columns A, C, G, T; every entry
 *               < n_states. State 0 is q0 and the target of the reset symbol.
 *   n_states    1 .. 2^24.
 *   accept_mask host, bit-packed: bit (q % 8) of byte q / 8 set <=> q in F;
 *               ceil(n_states / 8) bytes.
 *   out         receives the handle; the library owns it until dfa_free.
 * The table is copied (the caller may free its buffers on return). dfa_load also
 * analyses the automaton on the host (its definite depth: the smallest m such that
 * any m symbols bring every state to one state, when m <= 64; and, for automata of at
 * most 256 states that are not definite, whether runs from all states meet within 16
 * symbols of random DNA) and picks the speculation lookback, the table placement and
 * whether scans use chunk maps (DNA_PLACE_MAP).
 * Errors: DNA_ERR_INVALID_ARG, DNA_ERR_NOMEM, DNA_ERR_CUDA, DNA_ERR_NO_DEVICE.
 */
int dfa_load(const uint32_t *table, uint32_t n_states, const uint8_t *accept_mask,
             dna_dfa **out);

/*
 * dfa_load_labeled -- dfa_load for an automaton that recognises several patterns at
 * once and says which of them ends at each step. Alg. 1 of the paper keeps one counter
 * per accepting state of its regex-dna automaton (the switch into final_states[] and
 * the CR result struct) so that one scan gives a count per expression of Table V; here
 * each state carries the set of patterns it reports.
 *   table     as dfa_load.
 *   labels    host uint32 [n_states]: bit i of labels[q] set <=> pattern i ends when a
 *             step lands in q. F is the set of states with a non-zero mask.
 *   n_labels  number of patterns, 1 .. 32; every mask must fit in n_labels bits.
 * Every scan entry point accepts the handle (counting steps that land in F, whatever
 * their labels); dna_scan_labels also reports per-label counts and label masks.
 * Errors: as dfa_load; DNA_ERR_INVALID_ARG for a mask outside n_labels bits.
 */
int dfa_load_labeled(const uint32_t *table, uint32_t n_states, const uint32_t *labels,
                     uint32_t n_labels, dna_dfa **out);

/* dfa_free -- releases a handle (NULL is ignored). No scan using it may be in flight. */
void dfa_free(dna_dfa *dfa);

typedef struct {
    uint32_t n_states;
    int32_t  definite_depth;   /* m, or -1 when not m-definite for any m <= 64 */
    uint32_t lookback;         /* symbols read before each chunk to speculate its start */
    uint32_t placement;        /* DNA_PLACE_* chosen for this automaton */
    uint32_t accept_start;     /* 1 when state 0 is in F */
    int32_t  device;
    uint32_t chunk_maps;       /* 1 when scans run every chunk from every state (see DNA_PLACE_MAP) */
    uint32_t n_labels;         /* pattern labels (dfa_load_labeled), 0 for dfa_load */
} dna_dfa_info;

#define DNA_PLACE_AUTO       0
#define DNA_PLACE_SMEM_PAIR  1  /* two-symbol table, one copy per lane, shared memory */
#define DNA_PLACE_SMEM_ONE   2  /* one-symbol table in shared memory */
#define DNA_PLACE_GLOBAL_ONE 3  /* one-symbol table in global memory (L2 resident) */
/* Chunk maps (automata of at most 256 states): each chunk is run from every state at once
 * (the possible starting states of Sec. III-A taken in full: up to 16 states as 4-bit
 * fields of one or two registers per lane, else a warp per 32 start states), and a join
 * composes the chunk maps in order. dfa_load picks it for automata whose runs
 * from different states do not meet within 16 symbols of random DNA (speculation would
 * rarely be repaired in the chunk's first bytes); it can also be requested through
 * dna_plan.placement. Larger automata whose runs never meet are scanned with speculation
 * and repair, which is exact but walks every chunk boundary in order. */
#define DNA_PLACE_MAP        4
/* Hot-state rows (automata of 91 .. 16383 states, too large for per-lane two-symbol
 * tables): two-symbol rows for the states a walk on random DNA visits most, as many as
 * fit in shared memory beside one-symbol rows of every state (16-bit entries); a lane
 * whose 4 symbols meet a state without a two-symbol row redoes them with one-symbol steps.
 * Measured slower than DNA_PLACE_SMEM_ONE on GB300; chosen only by a plan or by dfa_tune. */
#define DNA_PLACE_SMEM_HOT   5
/* One-symbol table copied once per lane in shared memory (512 B per state, so automata of
 * up to about 375 states): every lane reads its own bank, so lookups never conflict.
 * Measured slower than DNA_PLACE_SMEM_ONE on GB300 (the one-symbol scans are bound by the
 * dependent lookup chain and instruction issue, not by bank conflicts); chosen only by a
 * plan or by dfa_tune. */
#define DNA_PLACE_SMEM_ONE_REP 6

int dfa_info(const dna_dfa *dfa, dna_dfa_info *out);

/*
 * dfa_tune -- the autotuner of the table placement (the lookup stride and table form):
 * times every placement the automaton fits in (two-symbol copies per lane; one shared
 * one-symbol table; one-symbol copies per lane; hot-state two-symbol rows; the
 * one-symbol table in L2) on the caller's sample with CUDA events, three count-only
 * scans each, and makes the fastest the handle's default (dna_dfa_info.placement).
 * The paper's Sec. III-B.1 motivates one uniform cost per symbol; which table form
 * gives the lowest cost depends on the automaton and the hardware, so it is measured.
 *   seq, len   device sample (a few MiB to a few hundred MiB of typical input).
 *   out_placement  receives the chosen DNA_PLACE_* (DNA_PLACE_MAP for chunk-map
 *                  automata, which have no table placement to choose).
 *   out_ms     NULL, or receives the chosen placement's time per scan.
 * Synchronises 'stream'. Do not run it while scans of the same handle are in flight on
 * other streams. Errors: DNA_ERR_INVALID_ARG, DNA_ERR_CUDA, DNA_ERR_NOMEM.
 */
int dfa_tune(dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream,
             uint32_t *out_placement, float *out_ms);

/*
 * dfa_analyze -- host-only analysis of a table in the dfa_load layout (no GPU needed).
 * Writes the definite depth m (the smallest m such that every word of m symbols sends
 * all states to one state, so m symbols before a chunk fix its start state exactly;
 * Sec. III-B.3's converging point reached from every start), or -1 when the table is
 * not m-definite for any m <= 64 or has more than 4096 states (the analysis is
 * quadratic in the state count). Errors: DNA_ERR_INVALID_ARG, DNA_ERR_NOMEM.
 */
int dfa_analyze(const uint32_t *table, uint32_t n_states, int32_t *definite_depth);

/*
 * dna_scan -- scans one device sequence with one automaton (the plain path).
 *   seq            device pointer to len bytes (any alignment); may be NULL if len = 0.
 *   len            number of bytes (0 .. 2^40).
 *   stream         CUDA stream the work is queued on.
 *   out_count      device or host-mapped pointer; receives the exact count.
 *   out_positions  device pointer or NULL. When non-NULL, receives the first
 *                  min(count, positions_capacity) match positions (uint64, ascending).
 *                  A count above positions_capacity is visible as *out_count >
 *                  positions_capacity; the written positions are then the smallest
 *                  positions_capacity ones. (The call returns before the count exists
 *                  on the device, so it cannot return DNA_ERR_CAPACITY for this; the
 *                  synchronous dna_scan_host does.)
 *   positions_capacity  number of uint64 slots at out_positions.
 * Scratch: the call takes stream-ordered device scratch sized O(len / chunk) from a
 * memory pool the library keeps per device, and returns it on the same stream. The pool
 * keeps up to 1 GiB reserved between calls, so repeated calls map no new memory.
 * No kernel of a scan waits on another block or on the host, so no device-side error
 * can arise after the call returns except CUDA's own (reported by the stream).
 * Kernels: one chunk-scan kernel (speculation, chunk scan, join) and, with positions,
 * one extraction kernel; automata using chunk maps run a map kernel and a join kernel
 * first (and, with positions, a kernel giving every sub-chunk's start for automata of
 * at most 16 states, then the chunk-scan kernels from the exact chunk starts).
 * Errors: DNA_ERR_INVALID_ARG (synchronous), DNA_ERR_NOMEM, DNA_ERR_CUDA,
 * DNA_ERR_CAPACITY (a plan's placement the automaton does not fit).
 */
int dna_scan(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream,
             uint64_t *out_count, uint64_t *out_positions, uint64_t positions_capacity);

/*
 * dna_scan_from -- dna_scan of one piece of a longer sequence (Sec. III-B: a chunk of the
 * input scanned from a given start state; the join of Sec. III-B.4 composes pieces).
 *   start_state     the state the run is in before the piece's first byte (the caller's
 *                   numbering, as in the table given to dfa_load; 0 for a whole sequence).
 *                   The piece's first chunk starts there exactly; later chunks are
 *                   speculated and repaired as in dna_scan.
 *   out_last_state  device pointer or NULL; receives the state after the piece's last
 *                   byte (the caller's numbering), which is start_state for len = 0.
 *   out_count, out_positions, positions_capacity
 *                   as dna_scan: accepting steps inside the piece, and their positions
 *                   counted from the piece's first byte.
 * Scanning the pieces of a sequence in order, each from the last state of the one before
 * it, gives the whole sequence's count and, offset by each piece's start, its positions;
 * scanning a piece from a guessed state and rescanning it when the guess was wrong gives
 * the same (the multi-process join composes pieces that way).
 * Asynchronous like dna_scan. Errors: DNA_ERR_INVALID_ARG (start_state >= n_states), and
 * as dna_scan.
 */
int dna_scan_from(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, uint32_t start_state,
                  dna_stream_t stream, uint64_t *out_count, uint32_t *out_last_state,
                  uint64_t *out_positions, uint64_t positions_capacity);

/*
 * dna_scan_labels -- dna_scan with per-pattern results, for an automaton loaded with
 * dfa_load_labeled (Alg. 1's count per accepting state, reported per pattern, Table V).
 *   out_count         as dna_scan: steps that land in a state with any label.
 *   out_label_counts  device uint64 [n_labels]: element i = steps that land in a state
 *                     whose mask has bit i (a step reporting two patterns counts for
 *                     both). Zeroed by the call on 'stream' before the scan adds to it.
 *   out_positions     device or NULL: as dna_scan (ascending end positions, at most
 *                     positions_capacity written).
 *   out_pos_labels    device uint32 or NULL (needs out_positions): the label mask of
 *                     each written position, same index.
 * The per-label counts are exact whatever positions_capacity is: the extraction pass
 * walks every row that holds a match. Asynchronous like dna_scan.
 * Errors: DNA_ERR_INVALID_ARG (no labels on the handle, NULL outputs, out_pos_labels
 * without out_positions), and as dna_scan.
 */
int dna_scan_labels(const dna_dfa *dfa, const uint8_t *seq, uint64_t len, dna_stream_t stream,
                    uint64_t *out_count, uint64_t *out_label_counts, uint64_t *out_positions,
                    uint32_t *out_pos_labels, uint64_t positions_capacity);

/*
 * dna_scan_host -- dna_scan on a sequence in host memory, with host-memory results.
 *   seq_host        host pointer to len bytes (pinned memory copies fastest).
 *   count_host      host pointer: receives the count.
 *   positions_host  host pointer or NULL; receives the first min(count,
 *                   positions_capacity) positions, as dna_scan's out_positions.
 * The call copies the sequence to a device buffer it allocates on 'stream', scans it,
 * copies the results back and returns after the stream has finished them (it is
 * synchronous with respect to the host). Returns DNA_ERR_CAPACITY when the count
 * exceeds positions_capacity (count_host then holds the true count and the smallest
 * positions_capacity positions were written). Other errors as dna_scan, plus
 * DNA_ERR_NOMEM when the device buffer cannot be allocated.
 */
int dna_scan_host(const dna_dfa *dfa, const uint8_t *seq_host, uint64_t len, dna_stream_t stream,
                  uint64_t *count_host, uint64_t *positions_host, uint64_t positions_capacity);

/*
 * dna_scan_count_static -- the count of dna_scan, computed without allocating memory.
 *   Same arguments and result as dna_scan with out_positions = NULL. The paper has no
 *   counterpart: this entry point exists for callers that cannot let a library
 *   allocate device memory while they run -- for example a server that reserves all of
 *   the GPU's memory up front and hands out fixed buffers, or code that must not trigger
 *   the implicit synchronisation an allocation can cause. Instead of stream-ordered
 *   scratch, the scan uses one fixed 4 MiB array in device memory that the library
 *   declares at file scope; every GPU that loads the library holds it until the process
 *   exits.
 *   Limits: len <= 2^36 bytes (64 GiB); a length or automaton whose chunk bookkeeping
 *   would not fit in the 4 MiB array returns DNA_ERR_CAPACITY before any work is queued.
 *   Set-up: the first call on a device looks up the array's device address (with that
 *   device current) and keeps it for the life of the process; make that first call
 *   before any stream capture, and do not call this entry point again after a reset of
 *   the device (cudaDeviceReset), which reloads the library's device code and moves the
 *   array.
 *   Sharing: all calls use the same array, which keeps the previous call's contents;
 *   calls that overlap on the GPU (different streams, or no ordering between them)
 *   race on it and give wrong counts. Order the calls, e.g. issue them on one stream.
 *   No cudaMalloc, cudaFree or allocating library routine is called (the library's
 *   allocation counter, dna_profile_t.device_allocs, does not move).
 *   Automata that dna_scan runs with chunk maps (dna_dfa_info.chunk_maps) run the same
 *   chunk-map kernels here, with their per-chunk maps in the array.
 * Errors: DNA_ERR_INVALID_ARG, DNA_ERR_CAPACITY, DNA_ERR_CUDA.
 */
int dna_scan_count_static(const dna_dfa *dfa, const uint8_t *seq, uint64_t len,
                          dna_stream_t stream, uint64_t *out_count);

/*
 * Plan override for dna_scan_planned (tests sweep it: results must not depend on it).
 *   chunk_bytes    bytes per chunk (one chunk per GPU lane); multiple of 128, >= 128;
 *                  0 = automatic.
 *   lookback       symbols read before a chunk to speculate its start state
 *                  (1 = the paper's possible starting states from one symbol);
 *                  0 = automatic; at most 64.
 *   warps_per_cta  8, 16, 24 or 32 (8 or 16 with DNA_PLACE_SMEM_HOT); 0 = automatic.
 *   placement      DNA_PLACE_*; 0 = automatic. A placement the automaton does not fit
 *                  in returns DNA_ERR_CAPACITY.
 *   prefetch_tiles how many 128-byte tiles ahead each lane prefetches its chunk into L2;
 *                  0 = automatic, 255 = no prefetch, at most 64 otherwise.
 *   hot_rows       DNA_PLACE_SMEM_HOT only: use two-symbol rows for at most this many
 *                  states (the most visited first); 0 = as many as fit.
 */
typedef struct {
    uint32_t chunk_bytes;
    uint32_t lookback;
    uint32_t warps_per_cta;
    uint32_t placement;
    uint32_t prefetch_tiles;
    uint32_t hot_rows;
} dna_plan;

int dna_scan_planned(const dna_dfa *dfa, const uint8_t *seq, uint64_t len,
                     dna_stream_t stream, uint64_t *out_count, uint64_t *out_positions,
                     uint64_t positions_capacity, const dna_plan *plan);

/*
 * Batched path: the counts of every (sequence, automaton) pair of a batch, computed by
 * one persistent kernel after one ingest kernel (the chunked scan of Sec. III-A applied
 * to many inputs and many automata at once; the paper runs one automaton over one input).
 * Automata with a definite depth <= 64 (dfa_info) and at most ~90 states run in the
 * persistent kernel; the others are scanned with dna_scan, one call per pair, inside
 * the same queued work.
 *
 * dna_batch_create -- builds a reusable plan for a fixed set of automata and sequences.
 *   dfas     host array of n_dfas handles (all loaded on the current device).
 *   seqs     host array of n_seqs device pointers; lens host array of their lengths. The
 *            plan keeps the pointers: the sequences must stay allocated (their contents
 *            may change between runs) until dna_batch_free.
 *   opts     NULL for defaults, or:
 *              chunk_bases    chunk length in bases, a multiple of 512 (<= 131072);
 *                             0 = 4096, or the autotuner's choice;
 *              warps_per_cta  8, 16 or 24; 0 = the most that fit;
 *              autotune       1 = time each (chunk length, warps) candidate on the
 *                             batch's own data during create and keep the fastest
 *                             (only when chunk_bases and warps_per_cta are 0);
 *              use_graph      1 = dna_batch_run captures the queued work into a CUDA
 *                             graph on its first call for a given out_counts pointer
 *                             and replays it afterwards.
 *   stream   used for the set-up copies (and the autotuner's runs); create returns
 *            after they have finished.
 *   out      receives the plan; the library owns it until dna_batch_free.
 * The plan allocates device memory for the packed copy of the sequences (one 2-bit code
 * per base plus one flag byte per 512 bases, about 0.25 bytes per base).
 * Errors: DNA_ERR_INVALID_ARG, DNA_ERR_NOMEM, DNA_ERR_CUDA, DNA_ERR_CAPACITY.
 */
typedef struct {
    uint32_t chunk_bases;
    uint32_t warps_per_cta;
    uint32_t autotune;
    uint32_t use_graph;
} dna_batch_opts;

typedef struct dna_batch dna_batch; /* opaque */

int dna_batch_create(const dna_dfa *const *dfas, uint32_t n_dfas,
                     const uint8_t *const *seqs, const uint64_t *lens, uint32_t n_seqs,
                     const dna_batch_opts *opts, dna_stream_t stream, dna_batch **out);

/*
 * dna_batch_run -- queues the batch on 'stream'.
 *   out_counts  device uint64 [n_seqs][n_dfas], row-major; element (s, d) receives the
 *               count of automaton d over sequence s (the dna_scan count).
 * Asynchronous: the counts are valid once the stream has completed the work. Runs of
 * one plan must not overlap in time (they share the plan's packed copy).
 * Errors: DNA_ERR_INVALID_ARG (NULL, wrong device), DNA_ERR_CUDA, DNA_ERR_NOMEM.
 */
int dna_batch_run(dna_batch *batch, dna_stream_t stream, uint64_t *out_counts);

/* dna_batch_info -- the plan the batch runs with. */
typedef struct {
    uint32_t chunk_bases;      /* chunk length */
    uint32_t warps_per_cta;
    uint32_t grid;             /* persistent blocks */
    uint32_t groups_per_task;  /* chunk groups (one chunk per lane) per ticket */
    uint32_t n_fast;           /* automata in the persistent kernel */
    uint32_t n_slow;           /* automata scanned with dna_scan */
    uint64_t n_chunks;
    uint64_t packed_tiles;     /* 512-base tiles of the packed copy */
    uint32_t max_states;       /* largest automaton in the persistent kernel */
} dna_batch_info_t;

int dna_batch_info(const dna_batch *batch, dna_batch_info_t *out);

/* dna_batch_free -- releases a plan (NULL is ignored). No run of it may be in flight. */
void dna_batch_free(dna_batch *batch);

/*
 * dna_scan_batch -- one-shot form: dna_batch_create (default options), dna_batch_run,
 * then dna_batch_free once the stream has finished the work. Arguments as above. The
 * call returns after the counts are complete (it synchronises 'stream').
 * Errors: as dna_batch_create and dna_batch_run.
 */
int dna_scan_batch(const dna_dfa *const *dfas, uint32_t n_dfas,
                   const uint8_t *const *seqs, const uint64_t *lens, uint32_t n_seqs,
                   dna_stream_t stream, uint64_t *out_counts);

/*
 * Request loop (serving): scans of mixed sizes against resident automata, admitted
 * continuously. A server owns 'slots' CUDA streams, a device memory pool and a
 * dispatcher thread. Submitted requests wait in arrival order; the dispatcher admits
 * the head request once its arrival time has passed, a slot is free and the memory it
 * needs (its length rounded up to 4 KiB, plus 1 MiB of scan scratch) fits under
 * mem_cap_bytes. An admitted request copies its sequence to the device, runs the count
 * scan of dna_scan and copies the count back, all on its slot's stream, so requests
 * in different slots overlap on the device. The paper scans one input at a time; this
 * is the serving form of that scan (no paper counterpart).
 *
 * dna_server_create -- dfas: host array of n_dfas handles (loaded on the current
 *   device; they stay resident and must outlive the server). opts may be NULL:
 *   slots (default 8, at most 256) and mem_cap_bytes (default 40 GiB).
 */
typedef struct {
    uint32_t slots;
    uint64_t mem_cap_bytes;
} dna_server_opts;

typedef struct dna_server dna_server; /* opaque */

int dna_server_create(const dna_dfa *const *dfas, uint32_t n_dfas, const dna_server_opts *opts,
                      dna_server **out);

/*
 * dna_server_submit -- queues a scan of host_seq[0, len) with automaton 'dfa' (an index
 *   into the server's array). host_seq should be pinned host memory (a pageable buffer
 *   makes the copy synchronous and stalls the dispatcher); it must stay valid and
 *   unchanged until the request's completion is reported. arrival_ns = 0 means now;
 *   otherwise a dna_server_now_ns() time before which the request is not admitted
 *   (open-loop load generation). Returns the request id (>= 0) or a negative DNA_ERR_*.
 */
int64_t dna_server_submit(dna_server *server, const uint8_t *host_seq, uint64_t len, uint32_t dfa,
                          uint64_t arrival_ns);

/* A finished request. Times are dna_server_now_ns() values. */
typedef struct {
    int64_t  id;
    int32_t  status;      /* DNA_OK, or the request's error (DNA_ERR_CAPACITY when it can never fit the cap) */
    uint32_t dfa;
    uint64_t count;       /* the dna_scan count */
    uint64_t len;
    uint64_t arrival_ns;  /* scheduled (or submit) time */
    uint64_t admit_ns;    /* when the dispatcher queued its work */
    uint64_t done_ns;     /* when the dispatcher saw its work complete */
    float    h2d_us;      /* device time of the host-to-device copy */
    float    device_us;   /* device time of copy + scan + result copy */
} dna_completion;

/* dna_server_poll -- moves up to max finished requests to out, waiting up to timeout_ms
 * (0 = no wait, < 0 = until one finishes) when none is ready. Returns how many. */
int dna_server_poll(dna_server *server, dna_completion *out, uint32_t max, int32_t timeout_ms);

/* dna_server_drain -- waits until every submitted request has finished (timeout_ms < 0:
 * no limit). DNA_ERR_TIMEOUT when the limit passes first. */
int dna_server_drain(dna_server *server, int32_t timeout_ms);

typedef struct {
    uint64_t submitted, completed, queued;
    uint32_t in_flight, slots;
    uint64_t mem_in_use, mem_cap;
} dna_server_stats_t;

int dna_server_stats(dna_server *server, dna_server_stats_t *out);

/* dna_server_now_ns -- the server clock (steady, nanoseconds). */
uint64_t dna_server_now_ns(void);

/* dna_server_free -- finishes every queued request, stops the dispatcher and releases
 * the server. NULL is ignored. */
void dna_server_free(dna_server *server);

/*
 * dna_fasta_parse -- host FASTA ingest (no GPU needed). A record is a '>' header line
 * (the '>' at the start of a line) and the sequence lines after it; text before the
 * first header is an unnamed record. Line breaks (LF, CR LF), spaces and tabs are
 * dropped and each record's remaining bytes are appended, unchanged, to 'out': letters
 * keep their case and non-base letters (N, IUPAC codes) stay and act as reset symbols in
 * the scans. Records are concatenated without separators; scan each record's span (for
 * instance as one dna_batch with a pointer per record) so that no match crosses records.
 *   text, len      the file contents (host).
 *   out, cap       host buffer for the sequence bytes, or NULL with cap = 0 to size only.
 *   out_len        receives the number of sequence bytes.
 *   rec_off        NULL, or uint64 [rec_cap]: record r is out[rec_off[r], rec_off[r+1]);
 *                  needs n_records + 1 entries.
 *   hdr_span       NULL, or uint64 [2 * rec_cap]: record r's header text is
 *                  text[hdr_span[2r], hdr_span[2r+1]) (empty for an unnamed record).
 *   n_records      receives the number of records.
 * Returns DNA_ERR_CAPACITY when out or rec_off is too small (the counts are still set).
 * The paper reads GenBank FASTA files (Sec. IV-A); this is the matching ingest.
 */
int dna_fasta_parse(const char *text, uint64_t len, uint8_t *out, uint64_t cap, uint64_t *out_len,
                    uint64_t *rec_off, uint64_t *hdr_span, uint32_t rec_cap, uint32_t *n_records);

/* dna_status_string -- a static description of a status code. */
const char *dna_status_string(int status);

/*
 * Host pattern compilers (convenience; no GPU needed). They return the minimal
 * complete DFA of Sigma*.L with canonical breadth-first numbering (state 0 = start),
 * in the dfa_load layout. *table_out and *accept_out are allocated by the library;
 * release them with dna_free_host.
 *   dna_compile_regex: syntax A C G T (case-insensitive), '.', [classes], ( ), |,
 *     * + ? {n} {n,} {n,m}; a pattern matching the empty word is rejected.
 *   dna_compile_kmers: Aho-Corasick automaton of n base strings (Sec. II; the
 *     failure-free form of Sec. III-B.1), minimised the same way.
 * Errors: DNA_ERR_SYNTAX, DNA_ERR_EMPTY_WORD, DNA_ERR_INVALID_ARG, DNA_ERR_CAPACITY,
 * DNA_ERR_NOMEM.
 */
int dna_compile_regex(const char *pattern, uint32_t **table_out, uint8_t **accept_out,
                      uint32_t *n_states_out);
int dna_compile_kmers(const char *const *kmers, uint32_t n_kmers, uint32_t **table_out,
                      uint8_t **accept_out, uint32_t *n_states_out);
/* dna_compile_regex_set: one minimal automaton for n_patterns (1 .. 32) regexes, the
 * DFA of Sigma*.(L1 | ... | Ln) in which each state's label mask (labels_out, uint32 per
 * state, for dfa_load_labeled) has bit i set when pattern i ends at a step landing in it
 * (the paper scans the nine expressions of Table V with one automaton). States with
 * different masks are never merged. Errors as dna_compile_regex. */
int dna_compile_regex_set(const char *const *patterns, uint32_t n_patterns, uint32_t **table_out,
                          uint32_t **labels_out, uint32_t *n_states_out);
void dna_free_host(void *p);

/*
 * Profiling hooks (bench and tests). When enabled, every scan records CUDA events
 * around its chunk-scan kernel on the caller's stream; dna_profile_read synchronises
 * those events and returns the accumulated kernel time and the number of kernels
 * this library launched since the last reset.
 */
typedef struct {
    double   scan_kernel_ms;    /* summed duration of the chunk-scan kernel */
    uint64_t scan_kernel_calls;
    uint64_t kernel_launches;   /* all kernels launched by the library */
    double   emit_kernel_ms;    /* position extraction kernel */
    uint64_t emit_kernel_calls;
    double   batch_kernel_ms;   /* batched scan kernel (dna_batch_run / dna_scan_batch) */
    uint64_t batch_kernel_calls;
    double   ingest_kernel_ms;  /* batched ingest (2-bit packing) kernel */
    uint64_t ingest_kernel_calls;
    /* speculation statistics of the profiled chunk scans (Sec. III-A, III-B.3): */
    uint64_t conv_scans;        /* scans counted */
    uint64_t conv_chunks;       /* chunks */
    uint64_t conv_inblock;      /* chunks whose speculated start was wrong and whose runs met
                                   within their first 16 bytes (repaired in the block) */
    uint64_t conv_pending;      /* chunks whose runs did not meet there (repaired by the last block) */
    uint64_t conv_blockfirst;   /* first chunks of blocks joined with a wrong start */
    uint64_t conv_diverged;     /* repairs that changed a chunk's last state */
    uint64_t conv_cascade;      /* chunks re-walked by the cascade */
    /* device allocations the library has made since it was loaded (handles, plans and
       stream-ordered scratch; never reset): */
    uint64_t device_allocs;
} dna_profile_t;

void dna_profile_enable(int enable);
int  dna_profile_read(dna_profile_t *out, int reset);

/*
 * dna_lookup_peak -- measures the lookup throughput that bounds the scans (a measurement
 * hook for their rooflines; the paper has no counterpart). Every thread of one full
 * block per SM runs 8 chains of dependent 4-byte table lookups; the best of three timed
 * runs (CUDA events on 'stream', after a warm-up run) gives lookups per second:
 *   mode 0  shared memory, lane l reading only bank l (the per-lane table copies of the
 *           two-symbol and chunk-map kernels): no bank conflict;
 *   mode 1  shared memory, random entries of a 64 KiB table (the shared one-symbol table);
 *   mode 2  global memory, random entries of a 128 KiB table read with ordinary (L1
 *           cached) loads (the one-symbol table of automata too large for shared memory).
 * Synchronises 'stream'. Errors: DNA_ERR_INVALID_ARG, DNA_ERR_CUDA, DNA_ERR_NOMEM.
 */
int dna_lookup_peak(uint32_t mode, dna_stream_t stream, double *lookups_per_s);

#ifdef __cplusplus
}
#endif
#endif /* DNA_DFA_H */
