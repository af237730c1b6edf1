"""Reader for the worked-example fixtures in tests/golden/.

Each fixture is copied from the paper (the citation is in its header).  Node
names and label names are strings in the files; they are mapped to integers
here in order of first appearance, which changes nothing about partitions.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class Fixture:
    def __init__(self):
        self.node_names = []      # node name per id
        self.node_label = []      # int label per id
        self.edges = []           # (src id, label int, dst id)
        self.add_nodes = []       # (name, label int)
        self.add_edges = []       # (src name, label int, dst name)
        self.pids = {}            # level -> list of printed identifiers
        self.et = []              # (sId, eLabel, tId, pid_old) as printed
        self.nt = {}              # column -> values
        self._nlab = {}
        self._elab = {}

    def nlab(self, s):
        return self._nlab.setdefault(s, len(self._nlab))

    def elab(self, s):
        return self._elab.setdefault(s, len(self._elab))

    def node(self, name):
        return self.node_names.index(name)

    def coo(self, edges=None):
        edges = self.edges if edges is None else edges
        s = np.array([e[0] for e in edges], dtype=np.uint32)
        l = np.array([e[1] for e in edges], dtype=np.uint32)
        d = np.array([e[2] for e in edges], dtype=np.uint32)
        return s, d, l


def load(name, base=None):
    f = Fixture() if base is None else base
    with open(os.path.join(GOLDEN, name)) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].split()
            if not line:
                continue
            op, args = line[0], line[1:]
            if op == "node":
                f.node_names.append(args[0])
                f.node_label.append(f.nlab(args[1]))
            elif op == "edge":
                f.edges.append((f.node(args[0]), f.elab(args[1]), f.node(args[2])))
            elif op == "complete":
                names, lab = args[:-1], f.elab(args[-1])
                for a in names:
                    for b in names:
                        if a != b:
                            f.edges.append((f.node(a), lab, f.node(b)))
            elif op == "add_node":
                f.add_nodes.append((args[0], f.nlab(args[1])))
            elif op == "add_edge":
                f.add_edges.append((args[0], f.elab(args[1]), args[2]))
            elif op == "pid":
                f.pids[int(args[0])] = [int(x) for x in args[1:]]
            elif op == "et":
                f.et.append((args[0], args[1], args[2], int(args[3])))
            elif op.startswith("nt_"):
                f.nt[op[3:]] = [int(x) for x in args]
            else:
                raise ValueError("unknown fixture line: " + raw)
    return f


def canonical(values):
    """Relabel identifiers by order of first appearance (0, 1, 2, ...)."""
    m = {}
    return [m.setdefault(v, len(m)) for v in values]
