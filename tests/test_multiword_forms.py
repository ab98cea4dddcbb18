"""Traces longer than a word: the carries between a trace's words, derived from
the LTLf definitions and checked here by brute force (no GPU). The device code
applies exactly these forms per word (planes from the last to the first); the
GPU tests then compare its levels with the oracle's.

Within a word (n positions, position 0 in the top bit), given what holds just
after the word's last position (the first position of the next word):
  X: (a << 1) | top bit of the next word
  F: -(a & -a) | (all of the word's positions if any later word has a set bit)
  U: psi | (phi & (((phi | psi) + psi + cin) ^ (phi & ~psi))), cin = U at the
     next word's first position (0 after the last word)
"""
import itertools
import random

import numpy as np


def until_def(phi, psi, n, cin=0):
    out = 0
    for t in range(n):
        ok = False
        for j in range(t, n):
            if (psi >> (n - 1 - j)) & 1 and all((phi >> (n - 1 - k)) & 1 for k in range(t, j)):
                ok = True
                break
        if not ok and cin and all((phi >> (n - 1 - k)) & 1 for k in range(t, n)):
            ok = True
        if ok:
            out |= 1 << (n - 1 - t)
    return out


def until_carry(phi, psi, n, cin):
    m = (1 << n) - 1
    s = ((phi | psi) + psi + cin) & m
    return (psi | (phi & (s ^ (phi & ~psi & m)))) & m


def test_until_with_carry_in_equals_the_definition():
    n = 5
    for phi, psi, cin in itertools.product(range(1 << n), range(1 << n), (0, 1)):
        assert until_carry(phi, psi, n, cin) == until_def(phi, psi, n, cin), (phi, psi, cin)


def _split(x, n, words):
    return [(x >> (n * (words - 1 - w))) & ((1 << n) - 1) for w in range(words)]  # word 0 = earliest positions


def test_chained_until_future_next_equal_the_definition():
    rng = random.Random(7)
    for n, words in ((3, 2), (4, 3), (5, 4)):
        N = n * words
        for _ in range(4000):
            phi, psi, a = rng.getrandbits(N), rng.getrandbits(N), rng.getrandbits(N)
            P, S, A = _split(phi, n, words), _split(psi, n, words), _split(a, n, words)
            m = (1 << n) - 1
            # U: last word first, carry = U at the next word's first position
            r, c = [0] * words, 0
            for w in reversed(range(words)):
                r[w] = until_carry(P[w], S[w], n, c)
                c = r[w] >> (n - 1)
            whole = 0
            for w in range(words):
                whole = (whole << n) | r[w]
            assert whole == until_def(phi, psi, N)
            # F
            f = [((-(A[w] & -A[w])) & m) | (m if any(A[w + 1:]) else 0) for w in range(words)]
            fw = 0
            for w in range(words):
                fw = (fw << n) | f[w]
            assert fw == until_def((1 << N) - 1, a, N)
            # X
            x = [((A[w] << 1) & m) | ((A[w + 1] >> (n - 1)) if w + 1 < words else 0) for w in range(words)]
            xw = 0
            for w in range(words):
                xw = (xw << n) | x[w]
            assert xw == (a << 1) & ((1 << N) - 1)


def test_pack_traces_splits_long_traces_into_words():
    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn as L
    bits = np.zeros((2, 70, 2), dtype=bool)
    bits[0, 0, 0] = bits[0, 33, 0] = bits[0, 69, 1] = True
    bits[1, 40, 1] = True
    p = L.pack_traces(bits, np.array([70, 41], dtype=np.int32), 1, 1, 32)
    assert p.planes == 3 and p.atom_words.shape == (2, 2, 3)
    assert p.atom_words[0, 0, 0] == 1 and p.atom_words[0, 0, 1] == 2 and p.atom_words[1, 0, 2] == 1 << 5
    assert p.atom_words[1, 1, 1] == 1 << 8 and p.atom_words[0, 1].sum() == 0
