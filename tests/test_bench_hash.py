"""The source hash that ties the committed DRAM counters to the step-kernel code (bench.py):
edits to comments keep it, edits to code change it, and string literals survive the comment
removal (so `"//"` inside one is code)."""
import bench

SRC = '''// header comment
#include "a.cuh"
/* block
   comment */ int f(int x) { return x + 1; }  // trailing
const char *s = "not // a comment";
char c = '/';
'''


def test_comments_do_not_count():
    other = SRC.replace("// header comment", "// a longer header comment\n// over two lines")
    other = other.replace("/* block\n   comment */", "/* another block */")
    assert bench.strip_comments(other) == bench.strip_comments(SRC)


def test_code_and_literals_count():
    t = bench.strip_comments(SRC)
    assert 'int f(int x) { return x + 1; }' in t
    assert '"not // a comment"' in t
    assert "char c = '/';" in t
    assert "header" not in t and "trailing" not in t and "block" not in t
    assert bench.strip_comments(SRC.replace("x + 1", "x + 2")) != t
    assert bench.strip_comments(SRC.replace("not // a", "not /* a")) != t


def test_profiled_traffic_is_read_or_withheld():
    # the committed profile carries the hash of the code its counters were taken on; the bench
    # reports the traffic (at least the 2.55 GB of algorithmic bytes of a 256^3 launch) only
    # while the two agree, and None after a code change until the next capture
    got = bench.profiled_traffic()
    assert got is None or got > 2.5e9
