cd "$(dirname "$0")"
bash build3.sh
for v in a b c d e f; do echo "== $v"; ./sb_$v 3e8 5 seg || exit 1; done
