"""The autotuner's decisions on synthetic timings (no GPU): the kernel loop
unless a persistent form is faster by the margin, runs of equal choices
merged into n <= nmax entries, and a table the library's lookup reads."""
import re

from paper_1208_4869_gb300 import autotune as T


def test_choose_needs_the_margin():
    assert T.choose({(0, 0): 1.0, (1, 1): 0.99, (1, 2): 0.98, (1, 0): 0.985}) == (0, 0)
    assert T.choose({(0, 0): 1.0, (1, 1): 0.5, (1, 2): 0.6, (1, 0): 0.7}) == (1, 1)


def test_merge_and_table():
    picks = [(128, (1, 1)), (256, (1, 1)), (512, (1, 2)), (1024, (0, 0)), (2048, (0, 0))]
    e = T.merge(picks, 0, 2, "complex64 qmr")
    assert [(x[2], x[3], x[4]) for x in e] == [(256, 1, 1), (512, 1, 2), (1 << 62, 0, 0)]
    text = T.table_text(e, "test device")
    rows = re.findall(r"\{(-?\d+), (-?\d+), (\d+), (\d), (\d)\}", text)
    assert len(rows) == 3 and rows[0] == ("0", "2", "256", "1", "1")
    assert "kTune" in text and text.count("{") == text.count("}")
    empty = T.table_text([], "none")
    assert "{-1, -1, 0, 0, 0}" in empty
