"""Seeded synthetic inputs: Gaussian and spiked-model data matrices and raw start vectors.

This module is shared by the CPU oracle's tests, the GPU parity tests and ``bench.py``.
It holds none of the AM method's arithmetic: it only draws random numbers and builds
data matrices.  Start vectors are returned *raw* (i.i.d. N(0,1), not normalised);
normalising them is step "select initial point" of Algorithm 2 and each side does it
itself.

Generator (counter-based, identical on x86 and Arm up to libm rounding of log/cos):
  * SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014; constants as published by Vigna):
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
        z = (z ^ (z >> 27)) * 0x94D049BB133111EB
        z =  z ^ (z >> 31)
    word(key, i) = mix(key + (i + 1) * 0x9E3779B97F4A7C15), key = mix(seed ^ mix(stream))
  * uniform(key, i) = (word(key, i) >> 11) * 2**-53            in [0, 1)
  * Box-Muller (Box & Muller 1958): pair j uses u1 = 1 - uniform(2j), u2 = uniform(2j+1);
        z_{2j} = sqrt(-2 ln u1) cos(2 pi u2),  z_{2j+1} = sqrt(-2 ln u1) sin(2 pi u2)

Workloads (the paper's experiments use data we do not have; these synthetic stand-ins
have the shapes of its workloads):
  * ``gaussian_matrix``: A_ij ~ N(0,1)            (small dense case, n=100, p=500)
  * ``spiked_matrix``:   A = sum_k theta_k u_k v_k^T + N(0,1) noise, u_k Gaussian unit-norm,
                         v_k unit-norm with ``nnz`` nonzeros at random indices, N(0,1) values.
  * ``bag_of_words``:    a sparse document x word count matrix in compressed sparse rows, the
                         stand-in for the text corpora of Section 5 (word counts per article):
                         Zipf word popularity, log-normal document lengths, and a few planted
                         topics (small word sets that co-occur in a share of the documents).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 2.0 ** -53

# stream tags (arbitrary distinct constants) so that matrices, spikes and starts drawn
# from one user seed never share a counter range
STREAM_NOISE = 1
STREAM_SPIKE_U = 2
STREAM_SPIKE_V = 3
STREAM_SPIKE_IDX = 4
STREAM_STARTS = 5
STREAM_BOW_LEN = 6
STREAM_BOW_PERM = 7
STREAM_BOW_TOKENS = 8
STREAM_BOW_TOPIC = 9
STREAM_BOW_TOPIC_TOKENS = 10


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _mix(np.array([np.uint64(stream)], dtype=np.uint64))[0]
        return _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ s], dtype=np.uint64))[0]


def uniforms(key: np.uint64, start: int, count: int) -> np.ndarray:
    """uniform(key, i) for i in [start, start+count), float64 in [0, 1)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        w = _mix(key + i * _GOLDEN)
    return (w >> np.uint64(11)).astype(np.float64) * _TWO_M53


def normals(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Standard normals z_i, i in [start, start+count); ``start`` must be even."""
    if start % 2:
        raise ValueError("normals(): start must be even (Box-Muller pairs)")
    npairs = (count + 1) // 2
    u = uniforms(key, start, 2 * npairs)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = rad * np.cos(ang)
    z[1::2] = rad * np.sin(ang)
    return z[:count]


def _fill_normals(out: np.ndarray, key: np.uint64, chunk_rows: int = 256) -> None:
    """out.flat[i] = z_i (row-major), generated in row chunks to bound host memory."""
    rows, cols = out.shape
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        first = r0 * cols
        even = first - (first % 2)
        z = normals(key, even, (r1 - r0) * cols + (first - even))
        out[r0:r1] = z[first - even:].reshape(r1 - r0, cols)


def gaussian_matrix(n: int, p: int, seed: int, dtype=np.float64) -> np.ndarray:
    """A (n x p, row-major) with i.i.d. N(0,1) entries."""
    A = np.empty((n, p), dtype=dtype)
    _fill_normals(A, stream_key(seed, STREAM_NOISE))
    return A


def spike_components(n: int, p: int, k: int, nnz: int, seed: int):
    """(U, V): U n x k Gaussian unit columns, V p x k unit columns with ``nnz`` nonzeros."""
    U = normals(stream_key(seed, STREAM_SPIKE_U), 0, n * k).reshape(k, n).T.copy()
    U /= np.linalg.norm(U, axis=0)
    V = np.zeros((p, k))
    kidx = stream_key(seed, STREAM_SPIKE_IDX)
    vals = normals(stream_key(seed, STREAM_SPIKE_V), 0, k * nnz).reshape(k, nnz)
    nz = min(nnz, p)
    for c in range(k):
        # random indices without replacement: order of p i.i.d. uniforms
        order = np.argsort(uniforms(kidx, c * p, p), kind="stable")
        V[order[:nz], c] = vals[c, :nz]
        V[:, c] /= np.linalg.norm(V[:, c])
    return U, V


def spiked_matrix(n: int, p: int, thetas, nnz: int, seed: int, dtype=np.float32) -> np.ndarray:
    """A = sum_k theta_k u_k v_k^T + N(0,1) noise (n x p, row-major)."""
    thetas = np.asarray(thetas, dtype=np.float64)
    A = np.empty((n, p), dtype=dtype)
    _fill_normals(A, stream_key(seed, STREAM_NOISE))
    U, V = spike_components(n, p, len(thetas), nnz, seed)
    for r0 in range(0, n, 512):
        r1 = min(n, r0 + 512)
        blk = A[r0:r1].astype(np.float64)
        blk += (U[r0:r1] * thetas) @ V.T
        A[r0:r1] = blk.astype(dtype)
    return A


def spiked_thetas(n: int, p: int, base=(40.0, 30.0, 20.0, 15.0, 10.0)) -> np.ndarray:
    """theta_k = base_k * sqrt(n) / sqrt(p) (the spiked workloads' signal strengths)."""
    return np.asarray(base, dtype=np.float64) * np.sqrt(n) / np.sqrt(p)


def raw_starts(p: int, r: int, seed: int, dtype=np.float64) -> np.ndarray:
    """r raw Gaussian start vectors, shape (r, p) (one start per row), NOT normalised."""
    X = np.empty((r, p), dtype=dtype)
    _fill_normals(X, stream_key(seed, STREAM_STARTS))
    return X


def bag_of_words(n: int, p: int, nnz: int, seed: int, topics: int = 5, topic_words: int = 10,
                 topic_share: float = 0.08, zipf: float = 1.0, chunk_docs: int = 8192):
    """A sparse n x p word-count matrix (documents x words) in compressed sparse rows.

    Returns (indptr int64 [n+1], indices int32 [nnz'], data float32 [nnz']) with columns
    ascending within each row and no repeated column; nnz' is close to ``nnz``.

    Recipe (every draw counter-based, so any document range can be built on its own):
      * word popularity: Zipf, weight 1 / (rank + 1)**zipf, ranks given to the word ids by a
        random permutation (the vocabulary order of a corpus does not follow frequency);
      * document i draws m_i words with replacement from the popularity law, m_i log-normal
        (sigma 0.5) with a mean of 1.35 nnz / n draws (repeated draws merge into counts);
      * ``topics`` planted topics, each ``topic_words`` words of popularity rank in [50, 2000);
        a document belongs to topic t with probability ``topic_share`` (else to none) and then
        draws round(0.25 m_i) more words uniformly from that topic's words;
      * A[i, j] = the number of times document i drew word j.
    """
    n, p = int(n), int(p)
    mean_draws = 1.35 * nnz / n
    z = normals(stream_key(seed, STREAM_BOW_LEN), 0, n)
    m = np.maximum(1, np.rint(mean_draws * np.exp(0.5 * z - 0.125))).astype(np.int64)
    perm = np.argsort(uniforms(stream_key(seed, STREAM_BOW_PERM), 0, p), kind="stable")  # rank -> word
    w = 1.0 / np.power(np.arange(1, p + 1, dtype=np.float64), zipf)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    lo, hi = min(50, p - 1), min(2000, p)
    tk = stream_key(seed, STREAM_BOW_TOPIC)
    twords = np.empty((topics, topic_words), dtype=np.int64)
    for t in range(topics):
        ranks = lo + np.argsort(uniforms(tk, t * (hi - lo), hi - lo), kind="stable")[:topic_words]
        twords[t] = perm[ranks]
    u_topic = uniforms(tk, topics * (hi - lo), n)
    topic = np.where(u_topic < topics * topic_share, np.minimum((u_topic / topic_share).astype(np.int64),
                                                                  topics - 1), -1)
    extra = np.where(topic >= 0, np.rint(0.25 * m), 0).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(m)])
    eoff = np.concatenate([[0], np.cumsum(extra)])
    kt, ke = stream_key(seed, STREAM_BOW_TOKENS), stream_key(seed, STREAM_BOW_TOPIC_TOKENS)
    indptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for d0 in range(0, n, chunk_docs):
        d1 = min(n, d0 + chunk_docs)
        cnt = int(off[d1] - off[d0])
        doc = np.repeat(np.arange(d0, d1, dtype=np.int64), m[d0:d1])
        word = perm[np.minimum(np.searchsorted(cdf, uniforms(kt, int(off[d0]), cnt), side="right"), p - 1)]
        ecnt = int(eoff[d1] - eoff[d0])
        if ecnt:
            edoc = np.repeat(np.arange(d0, d1, dtype=np.int64), extra[d0:d1])
            pick = np.minimum((uniforms(ke, int(eoff[d0]), ecnt) * topic_words).astype(np.int64), topic_words - 1)
            doc = np.concatenate([doc, edoc])
            word = np.concatenate([word, twords[topic[edoc], pick]])
        keys, counts = np.unique(doc * p + word, return_counts=True)
        rows = keys // p
        cols.append((keys - rows * p).astype(np.int32))
        vals.append(counts.astype(np.float32))
        indptr[d0 + 1:d1 + 1] = np.cumsum(np.bincount(rows - d0, minlength=d1 - d0))
        indptr[d0 + 1:d1 + 1] += indptr[d0]
    return indptr, np.concatenate(cols), np.concatenate(vals)
