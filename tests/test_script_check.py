"""The edit-script checker used by the GPU edit-script tests, pinned on
scripts written out by hand (textbook kitten -> sitting, distance 3) and on
mistakes it must reject."""
import numpy as np

from script_check import DEL, INS, SUB, script_transforms


def b(s):
    return np.frombuffer(s.encode(), dtype=np.uint8)


def test_kitten_sitting():
    # k->s at 0, e->i at 4, insert g at the end
    ops = [(SUB, 0, 0), (SUB, 4, 4), (INS, 6, 6)]
    assert script_transforms(b("kitten"), b("sitting"), ops)


def test_rejects_wrong_scripts():
    A, B = b("kitten"), b("sitting")
    assert not script_transforms(A, B, [(SUB, 0, 0), (SUB, 4, 4)])              # g missing
    assert not script_transforms(A, B, [(SUB, 0, 0), (SUB, 3, 4), (INS, 6, 6)])  # misplaced
    assert not script_transforms(A, B, [(SUB, 4, 4), (SUB, 0, 0), (INS, 6, 6)])  # out of order
    assert not script_transforms(A, B, [(7, 0, 0), (SUB, 4, 4), (INS, 6, 6)])    # unknown kind


def test_deletions_insertions_and_empty():
    assert script_transforms(b("abc"), b(""), [(DEL, 0, 0), (DEL, 1, 0), (DEL, 2, 0)])
    assert script_transforms(b(""), b("xy"), [(INS, 0, 0), (INS, 0, 1)])
    assert script_transforms(b("same"), b("same"), [])
    assert not script_transforms(b("same"), b("sane"), [])
    # a deletion and an insertion in place of a substitution: valid, just longer
    assert script_transforms(b("ab"), b("xb"), [(DEL, 0, 0), (INS, 1, 0)])
