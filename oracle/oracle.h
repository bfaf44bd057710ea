/*
 * oracle.h -- plain, slow, single-threaded CPU oracle for the levelwise
 * wavelet-tree / wavelet-matrix construction of Shun, "Improved Parallel
 * Construction of Wavelet Trees and Rank/Select Structures".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path (the CUDA library,
 * its Python binding) may include, link, load or call this code.  Only the
 * test suite, the smoke check and the bench's CPU-baseline leg use it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Every function computes the plain definition of what the paper specifies
 * (cited per function), with no blocking, fusion or reordering.  All
 * arithmetic is integer.
 *
 * Conventions (each a reading of a passage that is silent on it):
 *   L(sigma)   = ceil(log2 sigma) levels, and 1 when sigma == 1.
 *   bit(x, k)  = (x >> k) & 1.  Level l tests bit(x, L-1-l): MSB first (§2).
 *   A level bitmap of nb bits is stored in u64 words, bit i at word i/64,
 *   bit i%64 (LSB first), padded with zero bits to a multiple of 2048 bits:
 *   orc_level_words(nb) = ceil(nb/2048)*32 words per level, levels stored
 *   back to back.
 */
#ifndef WT_ORACLE_H
#define WT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

uint32_t orc_levels(uint32_t sigma);
uint64_t orc_level_words(uint64_t nbits);

/* Balanced binary wavelet tree, levelwise and pointer-free (§2 definition,
 * pointer removal as in §2's space paragraph).  bits: L*orc_level_words(n). */
int orc_wt_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* bits);

/* Wavelet matrix (§4.3, wavelet-matrix paragraph).  bits as above;
 * zeros[L] = number of 0 bits of each level. */
int orc_wm_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* bits,
                 uint64_t* zeros);

/* Jacobson-style rank directory (§5.1 rank) with the fixed geometry
 * 2048-bit superblocks / 512-bit blocks.  rec has 2*(ceil(nbits/2048)+1) u64:
 * rec[2s]   = zeros in bits [0, 2048s)                    (counted bits < nbits)
 * rec[2s+1] = rel[0] | rel[1]<<16 | rel[2]<<32 | rel[3]<<48,
 *             rel[b] = zeros in [2048s, min(2048s+512b, nbits)).
 * The trailing record holds the level total and rel = 0. */
void orc_rank_dir(const uint64_t* bits, uint64_t nbits, uint64_t* rec);

/* Sampled select (§5.1 select, every 4096th occurrence kept): samp[k] =
 * position of the occurrence of bit value b with 0-based index 4096k, for
 * k < ceil(count_b/4096).  Returns the number of samples written. */
uint64_t orc_select_samples(const uint64_t* bits, uint64_t nbits, uint32_t b,
                            uint64_t* samp);

/* Constant-time select directory after Clark (§5.1 select: positions of
 * every k-th occurrence define ranges; long ranges store all answers,
 * short ones are sampled again into sub-ranges, long sub-ranges store all
 * answers, short ones are searched within a bounded span).  Fixed here for
 * 64-bit words: ranges of 4096 occurrences (the select samples), 16
 * sub-ranges of 256 occurrences per range; a range of at least huge_min
 * bits stores the absolute positions of its 4096 occurrences; a sub-range of
 * at least sparse_min bits stores the offsets (from its range's start) of
 * its 256 occurrences.  For occurrences of bit value b:
 *   desc[k]   range k: huge: 2^63 | 4096 * (huge ranges before k);
 *             else (sparse sub-ranges in earlier non-huge ranges) |
 *             (16-bit mask of its sparse sub-ranges) << 40
 *   sub[16k+i] offset of occurrence 4096k+256i from the range's start
 *             (0xffffffff past the last occurrence; 0 in huge ranges)
 *   sparse[256s+j] offset from its range's start of occurrence j of the
 *             s-th sparse sub-range (0xffffffff past the last occurrence)
 *   huge[4096h+j]  position of occurrence j of the h-th huge range
 *             (UINT64_MAX past the last occurrence)
 * huge_min <= 2^32 keeps every stored offset within 32 bits.  Call with
 * NULL arrays to get the three counts first.  Returns 0, or -1 when out of
 * memory. */
int orc_clark_build(const uint64_t* bits, uint64_t nbits, uint32_t b, uint64_t huge_min,
                    uint64_t sparse_min, uint64_t* nranges, uint64_t* nhuge, uint64_t* nsparse,
                    uint64_t* desc, uint32_t* sub, uint32_t* sparse, uint64_t* huge);

/* Generalized select for the digit levels of the 4-ary tree (§5.2: select
 * per character, by the same ranges and sub-ranges as the binary case):
 * the sampled and constant-time directories above, for the occurrences of
 * digit value d (0..3) in a digit level of ndig 2-bit digits; positions and
 * lengths count digits. */
uint64_t orc_digit_samples(const uint64_t* dig, uint64_t ndig, uint32_t d, uint64_t* samp);
int orc_clark_digits(const uint64_t* dig, uint64_t ndig, uint32_t d, uint64_t huge_min,
                     uint64_t sparse_min, uint64_t* nranges, uint64_t* nhuge, uint64_t* nsparse,
                     uint64_t* desc, uint32_t* sub, uint32_t* sparse, uint64_t* huge);

/* Huffman code lengths (§4.3 arbitrary-shaped trees; Huffman shape).
 * Heap keyed (weight, id), leaf id = symbol, internal id = sigma + creation
 * index; symbols with count 0 get length 0; a single present symbol gets
 * length 1.  If the longest code exceeds cap, lengths come from
 * package-merge limited to cap.  Returns the longest length. */
uint32_t orc_huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap,
                             uint8_t* len);
/* Canonical codes from lengths: sort by (len, symbol), consecutive values,
 * shifted left when the length grows.  code[s] holds len[s] bits. */
void orc_canonical_codes(const uint8_t* len, uint32_t sigma, uint32_t* code);
/* Level sizes n_l = #{i : len(S_i) > l}, l < maxlen. */
void orc_huff_level_sizes(const uint32_t* S, uint64_t n, const uint8_t* len,
                          uint32_t maxlen, uint64_t* nl);
/* Huffman-shaped wavelet tree: level l holds the elements with len > l,
 * stably ordered by their l-bit code prefix; the bit is code bit l, MSB
 * first.  Level l starts at word offset woff[l]. */
int orc_huff_wt_build(const uint32_t* S, uint64_t n, const uint8_t* len,
                      const uint32_t* code, uint32_t maxlen,
                      const uint64_t* woff, uint64_t* bits);

/* 4-ary wavelet tree (§4.3 multiary, d = 4): digit level beta keeps binary
 * level 2*beta of the balanced tree; its digit is bits
 * [L-1-2beta .. max(L-2-2beta, 0)] of the symbol (1 bit wide on the last
 * level when L is odd).  2 bits per digit, 32 digits per u64, LSB first,
 * orc_level_words(2*n) words per digit level. */
int orc_mwt_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* dig);
/* Per-digit rank directory (§5.2 generalized rank; per-value counts):
 * 8 u64 per 1024-digit superblock, plus a trailing total record.
 * rec[8s+v] (v<4) = count of value v in digits [0, 1024s);
 * rec[8s+4+b] = four u16 counts of values 0..3 in [1024s, 1024s+256b). */
void orc_mwt_dir(const uint64_t* dig, uint64_t ndig, uint64_t* rec);

/* Queries by their definitions on S (§2): access(S,i) = S[i];
 * rank_c(S,i) = #c in S[0..i] (inclusive); select_c(S,k) = position of the
 * k-th (1-based) occurrence.  Invalid arguments give UINT64_MAX. */
void orc_access(const uint32_t* S, uint64_t n, const uint64_t* i, uint64_t q,
                uint64_t* out);
void orc_rank(const uint32_t* S, uint64_t n, uint32_t sigma, const uint32_t* c,
              const uint64_t* i, uint64_t q, uint64_t* out);
void orc_select(const uint32_t* S, uint64_t n, uint32_t sigma, const uint32_t* c,
                const uint64_t* k, uint64_t q, uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif
