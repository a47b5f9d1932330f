"""Checks an edit script against the two strings it claims to transform
(test infrastructure; no test functions here).  A script is a sequence of
(kind, x, y): kind 0 puts B[y] in place of A[x], 1 deletes A[x], 2 inserts
B[y] before A[x]; the characters between two operations must match.  A
valid script with as many operations as the edit distance is optimal."""
import numpy as np

SUB, DEL, INS = 0, 1, 2


def script_transforms(A, B, ops) -> bool:
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    i = j = 0
    for kind, x, y in np.asarray(ops, dtype=np.int64).reshape(-1, 3):
        kind, x, y = int(kind), int(x), int(y)
        # matching characters from (i, j) up to the operation
        if x < i or y < j or x - i != y - j or not np.array_equal(A[i:x], B[j:y]):
            return False
        if kind == SUB:
            if x >= len(A) or y >= len(B):
                return False
            i, j = x + 1, y + 1
        elif kind == DEL:
            if x >= len(A):
                return False
            i, j = x + 1, y
        elif kind == INS:
            if y >= len(B):
                return False
            i, j = x, y + 1
        else:
            return False
    return len(A) - i == len(B) - j and np.array_equal(A[i:], B[j:])
