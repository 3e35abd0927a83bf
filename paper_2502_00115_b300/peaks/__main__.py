from paper_2502_00115_b300.peaks import run
import json

print(json.dumps(run()))
