"""Tune tables: the JSON form round-trips (no GPU needed)."""
from paper_1910_13555_gb300 import tune


def test_table_json_round_trip(tmp_path):
    table = {(5, 13): {"swap": 1, "ms": {0: 1.5, 1: 1.0}}, (23, 23): {"swap": 0, "ms": {0: 2.0, 1: 2.5}}}
    doc = tune.table_to_json(table, "GB300")
    back = tune.table_from_json(doc)
    assert {k: v["swap"] for k, v in back.items()} == {k: v["swap"] for k, v in table.items()}
    import json
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"GB300": doc}))
    assert json.loads(p.read_text())["GB300"]["entries"][0]["m"] == 5


def test_split_and_swap_tables_merge_and_round_trip():
    emu = {(5, 13): {"swap": 1, "ms": {0: 1.5, 1: 1.0}}}
    f64 = {(5, 13): {"split": 4, "ms": {1: 3.0, 4: 2.0}}, (13, 13): {"split": 1, "ms": {1: 1.0}}}
    both = tune.merge_tables(emu, f64)
    assert both[(5, 13)]["swap"] == 1 and both[(5, 13)]["split"] == 4
    assert "swap" not in both[(13, 13)] and both[(13, 13)]["split"] == 1
    back = tune.table_from_json(tune.table_to_json(both, "GB300"))
    assert back[(5, 13)]["swap"] == 1 and back[(5, 13)]["split"] == 4
    assert back[(13, 13)] == {"ms": back[(13, 13)]["ms"], "split": 1}
