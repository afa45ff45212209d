"""Summarise a parity log (JSON lines written by the GPU tests when PTYLM_PARITY_LOG is set)
as a markdown table: per test file, quantity, norm and bound, the number of cases, the worst
achieved error, the bound at that case and the largest error / bound ratio; for comparisons
against the independent FP32 evaluation also that evaluation's worst error.

    PTYLM_PARITY_LOG=parity.jsonl python -m pytest tests -m gpu
    python tests/parity_table.py parity.jsonl
"""
from __future__ import annotations

import json
import re
import sys
from collections import defaultdict


def load(path):
    with open(path) as fh:
        return [json.loads(line) for line in fh if line.strip()]


def quantity_key(q):
    # fold per-problem indices and lambda values so that one row covers a family
    q = re.sub(r"\[\d+\]", "[b]", q)
    return re.sub(r"\(G \+ [0-9.]+ ", "(G + lam ", q)


def table(records):
    groups = defaultdict(list)
    for r in records:
        test_file = r["test"].split("::")[0].split("/")[-1]
        groups[(test_file, quantity_key(r["quantity"]), r["norm"], r["basis"])].append(r)
    rows = ["| test file | quantity | norm | bound | cases | worst error | its bound | max error/bound | FP32-eval worst |",
            "|---|---|---|---|---|---|---|---|---|"]
    for (tf, q, norm, basis), rs in sorted(groups.items()):
        worst = max(rs, key=lambda r: r["err"])
        ratio = max(r["err"] / r["tol"] for r in rs)
        f32 = max((r.get("fp32_err", 0.0) for r in rs), default=0.0)
        rows.append(f"| {tf} | {q} | {norm} | {basis} | {len(rs)} | {worst['err']:.2e} | {worst['tol']:.2e} | "
                    f"{ratio:.2f} | {f32:.2e} |" if f32 else
                    f"| {tf} | {q} | {norm} | {basis} | {len(rs)} | {worst['err']:.2e} | {worst['tol']:.2e} | "
                    f"{ratio:.2f} | — |")
    return "\n".join(rows)


if __name__ == "__main__":
    print(table(load(sys.argv[1])))
