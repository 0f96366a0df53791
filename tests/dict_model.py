"""Non-private key-value semantics (Sec. 2.1): Get returns the value or null,
Put inserts or updates, Delete removes.  A plain Python dict applied op by op,
the stand-in for the paper's non-oblivious hash-table baseline (Sec. 5.3)."""
import numpy as np

GET, PUT, DEL = 0, 1, 2


class DictModel:
    def __init__(self, keys, vals):
        self.d = {int(k): bytes(v) for k, v in zip(keys, vals)}

    def apply(self, ops, keys, vals_in, val_bytes):
        n = len(ops)
        vout = np.zeros((n, val_bytes), dtype=np.uint8)
        status = np.zeros(n, dtype=np.uint8)
        zero = bytes(val_bytes)
        for i in range(n):
            k = int(keys[i])
            present = k in self.d
            status[i] = present
            if ops[i] == GET:
                vout[i] = np.frombuffer(self.d.get(k, zero), dtype=np.uint8)
            elif ops[i] == PUT:
                self.d[k] = bytes(vals_in[i])
            else:
                self.d.pop(k, None)
        return vout, status
