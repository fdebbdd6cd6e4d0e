"""Sequence database files.

read_fasta: a protein FASTA file (the form SwissProt ships in, Sec. III.B.5)
into the library's packed form -- one uint8 code stream (hs_encode's
24-symbol alphabet, unknown letters as X) and int64 offsets -- plus the
header lines.  save_db / load_db: the packed form as one .npz file, so a
large database is read and encoded once and reloaded without parsing.
"""
from __future__ import annotations

import gzip

import numpy as np

from . import encode


def read_fasta(path_or_lines):
    """(names, codes uint8, offsets int64[n+1]) from a FASTA file path
    (gzip-compressed when it ends in .gz) or an iterable of lines.  Sequence
    lines may wrap; blank lines are skipped; '*' stop codons inside a
    sequence are kept as letters (code 23); whitespace is dropped.  A file
    with no '>' header is one sequence named ''."""
    if isinstance(path_or_lines, str):
        lines = gzip.open(path_or_lines, "rt") if path_or_lines.endswith(".gz") else open(path_or_lines)
    else:
        lines = path_or_lines
    names, chunks, lengths = [], [], []
    cur = None
    try:
        for line in lines:
            line = line.rstrip("\r\n")
            if line.startswith(">"):
                if cur is not None:
                    s = "".join(cur)
                    chunks.append(s)
                    lengths.append(len(s))
                names.append(line[1:].strip())
                cur = []
            elif line.strip():
                if cur is None:
                    names.append("")
                    cur = []
                cur.append("".join(line.split()))
        if cur is not None:
            s = "".join(cur)
            chunks.append(s)
            lengths.append(len(s))
    finally:
        if isinstance(path_or_lines, str):
            lines.close()
    offsets = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=offsets[1:])
    text = "".join(chunks)
    codes = encode(text) if text else np.zeros(0, np.uint8)
    return names, codes, offsets


def save_db(path: str, codes, offsets, names=None):
    """The packed database (and optional names) as one compressed .npz."""
    extra = {} if names is None else {"names": np.asarray(names, dtype=object)}
    np.savez_compressed(path, codes=np.ascontiguousarray(codes, np.uint8),
                        offsets=np.ascontiguousarray(offsets, np.int64), **extra)


def load_db(path: str):
    """(codes, offsets, names or None) from save_db's file."""
    with np.load(path, allow_pickle=True) as z:
        names = z["names"].tolist() if "names" in z.files else None
        return z["codes"], z["offsets"], names
