"""FASTA reading and the packed database file (host only)."""
import gzip

import numpy as np

import oracle as O
from paper_1508_06561_gb300 import seqio


FASTA = """>sp|P1|ONE first protein
MKTAYIAKQR
QISFVKSHFS

>sp|P2|TWO
ACDEFGHIKLMNPQRSTVWY
>empty entry
>sp|P3|THREE with odd letters
MKU OJ*
"""


def test_read_fasta_packs_sequences_and_names():
    names, codes, offsets = seqio.read_fasta(FASTA.splitlines(True))
    assert names == ["sp|P1|ONE first protein", "sp|P2|TWO", "empty entry", "sp|P3|THREE with odd letters"]
    assert offsets.tolist() == [0, 20, 40, 40, 46]
    seqs = ["MKTAYIAKQRQISFVKSHFS", "ACDEFGHIKLMNPQRSTVWY", "", "MKUOJ*"]
    assert np.array_equal(codes, O.encode("".join(seqs)))
    assert codes[40 + 2] == O.encode("X")[0]            # unknown letters read as X


def test_headerless_file_and_empty_input():
    names, codes, offsets = seqio.read_fasta(["MKV\n", "LL\n"])
    assert names == [""] and offsets.tolist() == [0, 5]
    names, codes, offsets = seqio.read_fasta([])
    assert names == [] and len(codes) == 0 and offsets.tolist() == [0]


def test_save_and_load_roundtrip(tmp_path):
    path = str(tmp_path / "fa.fasta")
    with open(path, "w") as f:
        f.write(FASTA)
    names, codes, offsets = seqio.read_fasta(path)
    db = str(tmp_path / "db.npz")
    seqio.save_db(db, codes, offsets, names)
    c2, o2, n2 = seqio.load_db(db)
    assert np.array_equal(c2, codes) and np.array_equal(o2, offsets) and n2 == names
    seqio.save_db(db, codes, offsets)
    assert seqio.load_db(db)[2] is None


def test_gzip_fasta(tmp_path):
    path = str(tmp_path / "fa.fasta.gz")
    with gzip.open(path, "wt") as f:
        f.write(FASTA)
    plain = seqio.read_fasta(FASTA.splitlines(True))
    names, codes, offsets = seqio.read_fasta(path)
    assert names == plain[0] and np.array_equal(codes, plain[1]) and np.array_equal(offsets, plain[2])
