"""The paper's reported ratios (Sec. 6.2) and the algorithmic byte counts the
roofline figures divide by.  Host arithmetic only."""
from __future__ import annotations

import math


def compression_ratio(full_key_bits: int, distinction_bits: int) -> float:
    """Sec. 6.2: # full key bits / # distinction bits in keys."""
    return full_key_bits / distinction_bits


def full_sort_key_bytes(max_key_bytes: int, rid_bytes: int = 8, word: int = 8) -> int:
    """Sec. 6.2: full key + record id, in units of 8-byte words."""
    return math.ceil((max_key_bytes + rid_bytes) / word) * word


def compressed_sort_key_bytes(distinction_bits: int, rid_variant_bits: int, word: int = 8) -> int:
    """Sec. 6.2: distinction bits + variant bits of the record id, in 8-byte words."""
    return math.ceil((distinction_bits + rid_variant_bits) / (8 * word)) * word


def sort_key_ratio(full_bytes: int, compressed_bytes: int) -> float:
    return full_bytes / compressed_bytes


def radix_passes(nbits: int, digit_bits: int) -> int:
    return (nbits + digit_bits - 1) // digit_bits


def pass_bytes(n: int, ck_words: int) -> int:
    """One radix pass reads and writes every (compressed key, row id) pair."""
    return n * 2 * (4 * ck_words + 4)


def extract_bytes(n: int, key_bytes: int, ck_words: int) -> int:
    """Extraction reads every key once and writes its compressed key."""
    return n * (key_bytes + 4 * ck_words)


def extract_sort_alg_bytes(n: int, key_bytes: int, ck_words: int, passes: int) -> int:
    """Algorithmic bytes of extract + sort: W per key plus 2 (c + 4) per pass."""
    return n * key_bytes + passes * pass_bytes(n, ck_words)


def build_bytes(n: int, ck_words: int) -> int:
    """Leaf pass: reads sorted (ck, rid), writes rid (4 B) and D-bit (2 B)."""
    return n * (4 * ck_words + 4 + 4 + 2)


def perm_only_pass_arrays(ck_words: int, nbits: int, digit_bits: int) -> list:
    """(arrays read, arrays written) per pass of the permutation-only sort: a
    pass reads its digit word(s), the key words later passes still need and
    the row ids, and writes the still-needed words and the row ids."""
    out = []
    passes = radix_passes(nbits, digit_bits)
    for q in range(passes):
        shift = q * digit_bits
        wlo, bits = shift // 32, min(digit_bits, nbits - shift)
        straddle = (shift % 32) + bits > 32
        keep = ((q + 1) * digit_bits) // 32 if q + 1 < passes else ck_words
        read = {wlo} | ({wlo + 1} if straddle else set()) | set(range(keep, ck_words))
        out.append((len(read) + 1, len(range(keep, ck_words)) + 1))
    return out


def perm_only_sort_bytes(n: int, ck_words: int, nbits: int, digit_bits: int) -> int:
    """Algorithmic bytes of all passes of the permutation-only sort."""
    return sum(4 * n * (r + w) for r, w in perm_only_pass_arrays(ck_words, nbits, digit_bits))
